// pic_internal.h -- launchers shared by the translation units of libpic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic_device.cuh"

namespace pic {

// velocity bins of the marker sort key (cell, bin): bins_per_cell bins per cell of
// expected displacement, 16 per cell of it in all (displacements of +-8 cells a step;
// faster markers share the end bins).  Finer bins keep a warp's markers closer
// together after they move (fewer deposit-window misses): measured on C2 (48,828
// markers a cell) with sorting every second step, 64 quarter-cell bins 13.1 ms a step
// against 13.4 ms for 16 whole-cell bins.  With few markers a cell they buy nothing and
// the key count (M x bins) costs the single-block scan time, so sparse runs keep whole
// cells.
constexpr int kVelBinsBase = 16;
inline int bins_per_cell(long long np, int M) { return np >= 8192LL * M ? 4 : 1; }
// threads per block of the sweep kernels (two blocks per SM)
constexpr int kSweepThreads = 512;

// ---------------------------------------------------------------- particles
struct PartPtrs {
    int32_t *cell;      // cell index in [0, M)
    void *t;            // offset in [0,1): float or double
    void *p;            // momentum
    void *delta;        // subsystem-I iterate: displacement x^(k) - x^n, cell units
    void *pnew;         // subsystem-I iterate p^(k+1)
    int32_t *id;        // caller index of each stored marker
};

// Float staging images of the grid fields for the float-form sweeps, built on the
// grid side (prep kernels once per substep, solve epilogues once per sweep) so that
// the sweep blocks copy them instead of converting doubles per block range.  All
// pointers null in the double form.
struct StageImages {
    float2 *a;          // sweep I: fl(a_y / K!), fl(a_z / K!)
    float4 *f;          // sweep I: fl(ebar dx / S1), fl(a_j) - fl(a_{j-1}) for y and z, 0
    float2 *an;         // sweep II: fl(a^n / K!)
    float2 *ak;         // sweep II: fl(a^(k) / K!)
    float2 *lo;         // sweep II: fl((a^n/K! - an) + (a^(k)/K! - ak))
    double inv_fact;    // 1 / K!
    double escale;      // dx / S1 (S1: scale of the degree-(K-1) path means)
};

struct Sweep1Args {
    int M, H, Dlim, K, fp32;
    int acc;            // deposit window accumulator (ACC_*)
    long long np;
    double dx, dt, w;
    PartPtrs P;
    const double *ebar, *ga_y, *ga_z, *ay, *az;
    double *j;
    DevCtrl *ctrl;
    int warm;           // 1: delta^(0) = explicit predictor, computed in-kernel (first sweep)
    int first;          // 1: the first sweep of the loop (writes the start-point cache)
    // graph mode (the launch is replayed by a CUDA graph): the deposit buffer is
    // jpair[iter & 1], and the explicit warm start and the first-sweep role apply
    // when iter == 0, with iter read from ctrl at kernel start
    int graph;
    double *jpair[2];
    StageImages img;
    // start-point cache, 4 reals a marker (A_y(x^n), A_z(x^n), gamma(p^n, A(x^n)),
    // unused): written by the loop's first sweep, read by the later ones; NULL: none
    void *a0;
    // spin (double form, hbar != 0): spin components in caller order (indexed by id)
    double hbar;
    const double *sy, *sz;
};

struct Sweep2Args {
    int M, H, K, fp32;
    int acc;            // deposit window accumulator (ACC_*)
    long long np;
    double w;
    PartPtrs P;
    const double *an_y, *an_z, *ak_y, *ak_z;
    double *s_y, *s_z;
    int *status;        // error bits (STATUS_TIMEOUT)
    // graph mode: deposits go to sypair/szpair[iter & 1], iter read from ctrl
    int graph;
    const DevCtrl *ctrl;
    double *sypair[2], *szpair[2];
    StageImages img;
};

struct CurrentArgs {
    int M, H, Dlim, K, fp32;
    long long np;
    double dx, w;
    PartPtrs P;
    const double *disp;     // caller order, length units
    double *out;
    DevCtrl *ctrl;
};

struct DiagArgs {
    int M, K, fp32;
    long long np;
    double dx, w;
    PartPtrs P;
    const double *c0, *c1;  // field coefficients (gather: c0; kinetic: a_y, a_z)
    double *out;            // gather output (caller order) or rho
    double *acc;            // kinetic sum
    int Dlim;               // path gathers: largest displacement (cells)
    int *status;            // path gathers: error bits (STATUS_NUMERIC)
};

int launch_sweep1(const Sweep1Args &a, int grid, int block, size_t smem, cudaStream_t s);
// the predicted start of subsystem I: delta^(0) (explicit when a.warm) and its current
// into a.j; the sweep's launch shape and shared memory
int launch_predeposit(const Sweep1Args &a, int grid, int block, size_t smem, cudaStream_t s);
size_t sweep1_smem(int M, int H, int fp32);
int launch_sweep2(const Sweep2Args &a, int grid, int block, size_t smem, cudaStream_t s);
size_t sweep2_smem(int M, int H, int fp32);
int launch_current(const CurrentArgs &a, int grid, int block, size_t smem, cudaStream_t s);
int launch_charge(const DiagArgs &a, int grid, int block, size_t smem, cudaStream_t s);
size_t charge_smem(int M, int H);
int launch_gather(const DiagArgs &a, int field_degree, int grid, int block, cudaStream_t s);
int launch_gather_path(const DiagArgs &a, int grid, int block, cudaStream_t s);
int launch_kinetic(const DiagArgs &a, int grid, int block, cudaStream_t s);
int launch_finalize1(int fp32, long long np, int M, PartPtrs P, bool zero_delta, int grid, int block,
                     cudaStream_t s);
int launch_load(int fp32, long long np, int M, double dx, const double *x, const double *p,
                PartPtrs P, int grid, int block, cudaStream_t s);
int launch_store(int fp32, long long np, double dx, PartPtrs P, double *x, double *p,
                 int grid, int block, cudaStream_t s);
// the same values in caller order through an inverse permutation (inv: np int32 of
// scratch); consecutive writes, so x and p may be device addresses of page-locked host memory
int launch_store_ordered(int fp32, long long np, double dx, PartPtrs P, int32_t *inv, double *x, double *p,
                         int grid, int block, cudaStream_t s);
int sweep_blocks_per_sm(int K, int fp32, int acc, int which, int block, size_t smem);
// whether the sweep kernels are built for (degree, form, accumulator)
bool sweep_variant_ok(int K, int fp32, int acc);
// one run's counting sort in a batched launch (key: cell * nbins + velocity bin)
struct SortRun {
    long long np;
    int M, nbins;
    float taup;             // dt / dx times the bins per cell
    PartPtrs src, dst;
    int32_t *counts;        // 2 M nbins: histogram, then cursors
};
int launch_sort_ens(int fp32, const SortRun *runs, int nruns, int grid_x, cudaStream_t s);
int launch_sort(int fp32, long long np, int M, double tau, int per, PartPtrs src, PartPtrs dst,
                int32_t *counts, int grid, int block, cudaStream_t s);

// ---------------------------------------------------------------- grid
// FP32 form, subsystem I: the last field increment must be below this fraction of
// the field's max-norm.  The momenta of the last sweep were updated with the field
// of the sweep before, so the energy error of a step is proportional to that
// increment.  Started from e^n the field converges from one side and the error has
// one sign, step after step (a drift, measured 1e-12 of the energy a step on C2 at
// 1e-9): 1e-10 is needed.  Started from the field of the proposal (warm_field) the
// last increment's sign varies and 3e-9 leaves no drift.
constexpr double kFieldIncrementRel = 1e-10;
constexpr double kFieldIncrementRelPredicted = 3e-9;

// CONV_START1: e^(0) = e^n - M1^{-1} j^(0) and ebar^(0), without a convergence decision
enum ConvMode { CONV_PLAIN = 0, CONV_SOLVE1 = 1, CONV_SOLVE2 = 2, CONV_START1 = 3 };

struct ConvArgs {
    int M, d_start, ntap, mode, ncomp;
    const double *taps;
    const double *in[2];
    double *out[2];
    const double *en[2];    // e^n
    double *ek[2];          // e^(k) (in: previous, out: new)
    double *aux[2];         // SOLVE1: ebar out; SOLVE2: a^(k) out
    const double *an[2];    // SOLVE2: a^n
    const double *r0[2];    // SOLVE2: P^{-1} b
    double *zero[2];        // deposit buffers of the next sweep, cleared here
    double dt, dx, tol, dtol;
    double erel;        // FP32 subsystem I: field increment tolerance relative to the field's max-norm
    int max_iter, fp32, subsystem;
    DevCtrl *ctrl;
    // graph mode: in[c] = pair[c][iter & 1], zero[c] = pair[c][(iter + 1) & 1]
    // (iter read from ctrl at kernel start), and the decision sets the loop's
    // conditional handle (1 = run another sweep)
    int graph;
    double *pair[2][2];
    unsigned long long cond_handle;
    StageImages img;    // SOLVE1: f.x = ebar image; SOLVE2: ak, lo
    int *count;         // graph mode of single runs: sweeps counted by the decision (or NULL)
};

int launch_conv(const ConvArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- spin (double form)
// Spin components are kept in caller order (sx[id], sy[id], sz[id]).
struct SpinArgs {
    int M, K;
    long long np;
    double dx, w, dt, hbar;
    PartPtrs P;                 // markers in stored order (cell, t as double, id)
    const double *ay, *az;
    double *sx, *sy, *sz;
    double *dy, *dz;            // spin deposit outputs (M each)
    double *acc;                // Zeeman energy sum (without hbar)
};
// d_y,i = sum_a w s_y,a Lambda^1_i(x_a), d_z likewise (Lambda_1(X)^T W S of subsystem II)
int launch_spin_deposit(const SpinArgs &a, int grid, cudaStream_t s);
// subsystem III: exact rotation of every spin
int launch_spin_rotate(const SpinArgs &a, int grid, cudaStream_t s);
// *acc += sum_a w (s_y dA_z/dx - s_z dA_y/dx)(x_a)
int launch_spin_energy(const SpinArgs &a, int grid, cudaStream_t s);
// b_y -= dt hbar (G^T d_z), b_z += dt hbar (G^T d_y), (G^T v)_j = (v_j - v_{j+1}) / dx
int launch_spin_rhs(int M, double dx, double dt, double hbar, const double *dy, const double *dz,
                    double *by, double *bz, cudaStream_t s);
// raise the spin deposit's dynamic shared-memory limit for a grid of M cells
int spin_optin(int M);

// split runs: buf[0..2] = (max increment, numeric bit, timeout bit) of the control block
int launch_split_pack(const DevCtrl *c, double *buf, cudaStream_t s);
int launch_split_unpack(DevCtrl *c, const double *buf, cudaStream_t s);

// ---------------------------------------------------------------- batched ensemble
// Many independent runs advance together: one launch of each kernel covers every
// run.  The particle sweeps are persistent kernels that claim work items (a run
// and a range of item_markers of its markers) from a queue built before each
// sweep from the runs still iterating; grid-side kernels take one block row per run.
constexpr int kEnsMaxRuns = 1024;

struct EnsQueue {
    int next;                // claim counter of the current sweep
    int nitems;              // items of the current sweep
    int nactive;             // runs in the current sweep
    int n_decided;           // runs that took their convergence decision in this sweep
    int n_continue;          // ... and go on
    int go;                  // 1: some run goes on after this sweep
    int item_markers;        // markers per item (a multiple of the tile size)
    int nblocks;             // sweep blocks that claim items (the rest leave at once)
    int loops[2];            // sweeps of the loops of subsystems I and II (all runs together)
    int item_start[kEnsMaxRuns + 1];
    int active[kEnsMaxRuns];
};

struct EnsRun {
    long long np;
    DevCtrl *ctrl;
};

// per-run pointers of the grid-side kernels
// Field changes of the last solves of each subsystem (x: subsystem I's e_x; y, z:
// subsystem II's e_y, e_z): d[0] = e^n - e^{n-1}, d[1] = e^{n-1} - e^{n-2}, ...
// order1 / order2: the degree of the time extrapolation that starts each
// subsystem's iteration (0: e^(0) = e^n), at most kMaxStartOrder.
constexpr int kMaxStartOrder = 3;
struct FieldHist {
    double *x[kMaxStartOrder], *y[kMaxStartOrder], *z[kMaxStartOrder];
    int order1, order2;
};

struct RunDesc {
    int M, K, fp32;
    long long np;
    double dx, dt;
    PartPtrs P;
    double *ex, *ek, *ebar, *ay, *az, *ga_y, *ga_z, *j0, *j1;
    const double *rowPm, *rowK;
    double *ey, *ez, *by, *bz, *eky, *ekz, *aky, *akz, *sy0, *sz0, *sy1, *sz1;
    DevCtrl *ctrl;
    StageImages img;
    FieldHist fh;
};

int launch_ens_plan(EnsQueue *Q, const EnsRun *runs, int nruns, unsigned long long cond, cudaStream_t s);
int launch_ens_status(const EnsRun *runs, int nruns, int *status, cudaStream_t s);
int conv_ens_optin(int Mmax, int ntap_max);
int launch_conv_ens(const ConvArgs *runs, int nruns, int Mmax, int ncomp, int ntap_max, EnsQueue *Q,
                    int *sweeps, unsigned long long cond, cudaStream_t s);
int launch_prep1_ens(const RunDesc *R, int nruns, int Mmax, cudaStream_t s);
int launch_prep2_ens(const RunDesc *R, int nruns, int Mmax, cudaStream_t s);
int launch_commit_ens(const RunDesc *R, int nruns, int Mmax, int which, cudaStream_t s);
int launch_sweep1_ens(int K, int fp32, const Sweep1Args *runs, int nruns, EnsQueue *Q, int grid,
                      size_t smem, cudaStream_t s);
int launch_sweep2_ens(int K, int fp32, const Sweep2Args *runs, int nruns, EnsQueue *Q, int grid,
                      size_t smem, cudaStream_t s);
// the predicted start of every run in the queue (delta^(0) and its current into each run's a.j)
int launch_predeposit_ens(int K, int fp32, const Sweep1Args *runs, int nruns, EnsQueue *Q, int grid,
                          size_t smem, cudaStream_t s);
int launch_finalize1_ens(int fp32, const RunDesc *R, int nruns, int grid_x, cudaStream_t s);
int launch_prep1(const RunDesc &R, cudaStream_t s);
int launch_prep2(const RunDesc &R, cudaStream_t s);
// end of a substep (which = 1, 2): the converged iterate becomes the state, and
// its change is recorded for the next starting field
int launch_commit(const RunDesc &R, int which, cudaStream_t s);
// scale S of the scaled path means of degree d (the sweeps' piece_means_scaled)
int mean_scale(int d);
int launch_poisson_rhs(int M, double dx, const double *rho, double *d, cudaStream_t s);
int launch_energy_grid(int M, int K, double dx, const double *rowM0, const double *rowM1,
                       const double *rowK, const double *ex, const double *ey, const double *ez,
                       const double *ay, const double *az, const double *rho, double *diag,
                       cudaStream_t s);
int launch_ctrl_reset(DevCtrl *ctrl, cudaStream_t s);

// learned warm start (pic_mlp.cu)
struct WarmArgs {
    int M, K, fp32;
    long long np;
    double dx, dt;
    PartPtrs P;
    const double *ex, *ay, *az;
    const float *params, *norm;
    int *status;        // error bits (STATUS_TIMEOUT)
};
int launch_warm_mlp(const WarmArgs &a, int grid, cudaStream_t s);

// message returned by pic_last_error(NULL) on the calling thread
void set_thread_error(const char *msg);

// host-side spline algebra (exact rows and inverse taps of the circulant matrices)
void mass_band(int d, double dx, double *band /* d+1 */);
void inverse_taps(const double *band, int bw, int M, double cut, double *g_full /* M */,
                  int *d_start, int *ntap, double *taps /* M */);

}  // namespace pic
