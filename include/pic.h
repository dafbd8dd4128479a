/*
 * pic.h -- C ABI of libpic, the GB300 (sm_103a) implementation of the
 * particle side of the energy-conserving PIC scheme of Y. Li,
 * "Energy conserving particle-in-cell methods for relativistic
 * Vlasov--Maxwell equations of laser-plasma interaction" (arXiv:2203.06513),
 * one dimension, with or without spin (hbar).
 *
 * The discrete system (Sec. 3.1): M uniform periodic cells of width
 * dx = L/M; E_x in the degree-(k-1) spline space V1, E_y, E_z, A_y, A_z in
 * the degree-k space V0; N_p markers with positions x_a, momenta p_a and
 * equal weights w.  One time step is the Lie--Trotter composition of
 * subsystem I (x, p, e_x) and subsystem II (e_y, e_z, a_y, a_z) of Sec. 4.2,
 * each solved by fixed-point iteration of its discrete-gradient scheme.
 *
 * Conventions for every entry point:
 *  - Return value: PIC_OK (0) or an error code below; on error
 *    pic_last_error(h) returns a message owned by the handle (valid until the
 *    next call on that handle).  A NULL handle yields PIC_ERR_INVALID.
 *  - All floating-point arrays crossing the ABI are IEEE double, contiguous.
 *    Particle arrays have N_p entries and are in the caller's original marker
 *    order (the library may reorder markers internally and undoes it).  Grid
 *    arrays have M entries, index j = coefficient of the j-th basis function.
 *  - Arrays passed with mem = PIC_MEM_DEVICE are device pointers on the
 *    handle's device; with PIC_MEM_HOST they are host pointers (pageable or
 *    page-locked; pic_init's load kernel reads page-locked marker arrays over
 *    the host link itself and pic_get_state writes them the same way, while
 *    pageable ones are copied through device buffers).  The
 *    caller owns every array it passes; the handle never keeps a caller
 *    pointer after a call returns.
 *  - The handle owns its device state and scratch (allocated in pic_init,
 *    freed in pic_destroy).  They come from a stream-ordered memory pool that
 *    the library keeps per device: what pic_destroy returns stays reserved in
 *    that pool for later handles of the process (until the process exits), so
 *    a repeated pic_init does not map new device memory; other allocators of
 *    the process are not affected.  The stream must outlive the handle.
 *    All work is ordered on the stream given to
 *    pic_init (a cudaStream_t passed as void*; NULL = legacy default stream).
 *    Calls return after their results are complete on that stream unless
 *    stated otherwise.  A handle must not be used from two threads at once.
 */
#ifndef PIC_H_
#define PIC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PIC_OK              0
#define PIC_ERR_INVALID     1   /* bad argument or configuration            */
#define PIC_ERR_NOCONVERGE  2   /* fixed point hit max_iter; state is the last iterate */
#define PIC_ERR_CUDA        3   /* CUDA runtime error                        */
#define PIC_ERR_NOMEM       4   /* device or host allocation failed          */
#define PIC_ERR_NUMERIC     5   /* NaN/Inf or a displacement beyond c*dt     */

/* particle arithmetic */
#define PIC_FP64            0   /* particle state and arithmetic in double   */
#define PIC_FP32            1   /* particle state (cell, offset, p) and arithmetic in float;
                                   deposits accumulated, solves, convergence and energy in double */
/* memory spaces */
#define PIC_MEM_HOST        0
#define PIC_MEM_DEVICE      1

/* initial guess of the subsystem-I fixed point */
#define PIC_WARM_NONE       0   /* x^(0) = x^n                               */
#define PIC_WARM_EXPLICIT   1   /* x^(0) = x^n + dt p^n / gamma(p^n, A^n(x^n)) */
#define PIC_WARM_MLP        2   /* learned predictor loaded by pic_mlp_load  */

/* pic_deposit kinds */
#define PIC_DEP_CHARGE      0   /* rho_j = sum_a w Lambda^0_j(x_a)                                  */
#define PIC_DEP_CURRENT     1   /* j_i = sum_a w int_{x_a}^{x_a+d_a} Lambda^1_i  (d_a from aux)     */
#define PIC_DEP_SUSCEPT     2   /* s_i = sum_a w (A^n+A^*)(x_a) Lambda^0_i(x_a) / (g(p_a,A^n)+g(p_a,A^*)) */

/* pic_gather fields */
#define PIC_FIELD_EX        0   /* E_x,h(x_a) = sum_i e_x,i Lambda^1_i(x_a) */
#define PIC_FIELD_EY        1   /* E_y,h(x_a), V0                           */
#define PIC_FIELD_EZ        2
#define PIC_FIELD_AY        3   /* A_y,h(x_a), V0                           */
#define PIC_FIELD_AZ        4
#define PIC_FIELD_EX_PATHAVG 5  /* path mean of E_x,h along x_a -> x_a + d_a (see pic_gather) */

/* deposit accumulation (pic_config.deposit): how the sweeps of the FP32 form
 * sum the float contributions of the markers a lane holds before they reach the
 * double grid row.  The FP64 form always accumulates in double. */
#define PIC_ACC_DEFAULT      0  /* FP32: PIC_ACC_COMPENSATED                                  */
#define PIC_ACC_FLOAT        1  /* FP32, k = 3 or 5: plain float lane sums, float warp sums    */
#define PIC_ACC_COMPENSATED  2  /* FP32: compensated float pair per lane (two-sum), double warp sums */
#define PIC_ACC_DOUBLE       3  /* FP32, k = 3 or 5: double lane sums of the float contributions */

/* time splitting of pic_step (pic_config.splitting) */
#define PIC_SPLIT_LIE        0  /* Phi_II(dt) o Phi_I(dt), the paper's Lie--Trotter step (Sec. 5) */
#define PIC_SPLIT_STRANG     1  /* Phi_I(dt/2) o Phi_II(dt) o Phi_I(dt/2) (symmetric, second order) */

/* pic_substep selectors */
#define PIC_SUBSYSTEM_I     1
#define PIC_SUBSYSTEM_II    2
#define PIC_SUBSYSTEM_III   3   /* spin rotation (hbar != 0 only) */

typedef struct pic_handle pic_handle;

typedef struct {
    double  L;           /* domain length (periodic [0, L))                        */
    int32_t nx;          /* M: number of cells = dim V0 = dim V1, 8 <= M <= 8192;
                            the sweeps stage the whole periodic grid in shared
                            memory, so pic_init also rejects (PIC_ERR_INVALID)
                            grids whose staging exceeds it: about M + 2(k + dt/dx)
                            <= 4600 cells in the FP32 form, 4200 in FP64 (k = 5)  */
    int32_t degree;      /* k: degree of V0 (V1 has k-1), 2 <= k <= 5               */
    int64_t np;          /* N_p >= 1                                                */
    double  weight;      /* w: equal marker weight (L/N_p neutralises the background) */
    double  dt;          /* time step, 0 < dt, and dt/dx <= 64                      */
    double  tol;         /* fixed-point tolerance: max-norm of the position increment
                            (length units) and of the field increment               */
    int32_t max_iter;    /* cap on fixed-point sweeps per substep (1..1000)         */
    int32_t precision;   /* PIC_FP64 or PIC_FP32                                    */
    int32_t warm_start;  /* PIC_WARM_*                                              */
    int32_t sort_every;  /* re-sort markers by cell every this many steps (0: only at init) */
    int32_t deposit;     /* PIC_ACC_* (FP32 form; 0 = default)                      */
    int32_t splitting;   /* PIC_SPLIT_LIE or PIC_SPLIT_STRANG                       */
    double  hbar;        /* normalised Planck constant; nonzero turns the spin on
                            (FP64 form, Lie--Trotter steps, no learned warm start) */
    int32_t warm_field;  /* with a warm start: 1 = also start subsystem I's field from
                            the proposal, e^(0) = e^n - M1^{-1} j(x^n -> x^(0)), so that
                            the first sweep's kick uses a field consistent with x^(0)
                            (the fixed point is the same; only the sweep count changes) */
} pic_config;

/* FP64 arrays of the discrete state u = (X, P, S, e_x, e_y, e_z, a_y, a_z), Sec. 3.1.
 * Any member may be NULL where a call says it is ignored. */
typedef struct {
    double *x;           /* N_p positions in [0, L)        */
    double *p;           /* N_p longitudinal momenta       */
    double *ex;          /* M coefficients in V1           */
    double *ey, *ez;     /* M coefficients in V0           */
    double *ay, *az;     /* M coefficients in V0           */
    double *sx, *sy, *sz;/* N_p spin components (read and written only when hbar != 0) */
} pic_arrays;

/* Create a handle and load the initial state (Sec. 3.1).  Reads x, p, ey, ez,
 * ay, az (and sx, sy, sz when hbar != 0) from `in` (mem space `mem`); in->ex is
 * ignored: e_x is computed from
 * the discrete Poisson equation G^T M1 e_x = -Lambda_0(X)^T W 1 + dx 1 with
 * sum_j e_x,j = 0 (Remark 2 of Sec. 4.2, with the neutralising background).
 * Markers are sorted by cell.  On success *out owns the handle. */
int pic_init(const pic_config *cfg, const pic_arrays *in, int32_t mem,
             void *stream, pic_handle **out);

/* ---------------------------------------------------------------------
 * One plasma split over several processes by markers (one GPU each): the
 * markers are independent given the fields, and the fields couple them only
 * through sums over markers (Sec. 4.2).  Each process creates its handle
 * with pic_init_split on its own markers (cfg->np = the local count, weight =
 * the global L / N_p) and the same initial fields; every later call is made on
 * every process in the same order.  The library then passes every sum over
 * markers that the fields need -- the charge of the discrete Poisson equation,
 * each sweep's current (subsystem I) and susceptibility (subsystem II) deposit,
 * the spin source, the kinetic, Zeeman and Gauss sums of pic_energy -- and the
 * fixed-point test's largest marker increment with the error bits through
 * reduce(ctx, op, buf, n, stream): buf is a device array of n doubles ordered on
 * `stream` (the handle's); the callback must replace it, in stream order, by the
 * elementwise sum (op = PIC_REDUCE_SUM) or max (PIC_REDUCE_MAX) over all
 * processes -- an all-reduce such as ncclAllReduce on that stream -- and return
 * 0 (nonzero: the call fails with PIC_ERR_CUDA).  Every process then solves the
 * same grid equations and takes the same decisions.  pic_deposit and pic_gather
 * act on the local markers only.  Split runs drive their loops from the host.
 * With reduce = NULL pic_init_split is pic_init.
 * --------------------------------------------------------------------- */
#define PIC_REDUCE_SUM      0
#define PIC_REDUCE_MAX      1
typedef int (*pic_reduce_fn)(void *ctx, int32_t op, double *buf, int64_t n, void *stream);

int pic_init_split(const pic_config *cfg, const pic_arrays *in, int32_t mem, void *stream,
                   pic_reduce_fn reduce, void *ctx, pic_handle **out);

/* Copy the current state to `out` (members that are NULL are skipped), in
 * the caller's marker order.  Positions are returned wrapped into [0, L). */
int pic_get_state(pic_handle *h, const pic_arrays *out, int32_t mem);

/* Deposit on the grid at the current positions (device output, `out`):
 *  PIC_DEP_CHARGE : out[M]   = rho (Lambda^0 deposit), aux ignored.
 *  PIC_DEP_CURRENT: out[M]   = w * path integral of Lambda^1 along x_a -> x_a + d_a
 *                   (Sec. 4.2, subsystem I), aux = device d[N_p] in caller order.
 *  PIC_DEP_SUSCEPT: out[2M]  = (s_y, s_z) of subsystem II (Sec. 4.2) with A^n the
 *                   handle's a and A^* from aux = device (a*_y[M], a*_z[M]).
 * Accumulation is in double. */
int pic_deposit(pic_handle *h, int32_t kind, const double *aux, double *out);

/* Gather a field at the current positions: out[N_p] (device), caller order.
 * PIC_FIELD_EX_PATHAVG: on entry out[a] holds a displacement d_a (length units,
 * |d_a| within the handle's halo, about dt + 2 dx); on return out[a] is the
 * path mean of E_x,h over the straight path x_a -> x_a + d_a, i.e.
 * (1/d_a) int Lambda^1(xi) dxi . e_x (Sec. 4.2, subsystem I), and E_x,h(x_a)
 * where d_a = 0.  Evaluated in double in both forms.  PIC_ERR_NUMERIC when a
 * displacement is not finite or beyond the halo. */
int pic_gather(pic_handle *h, int32_t field, double *out);

/* Advance one subsystem by dt (Sec. 4.2).  which = PIC_SUBSYSTEM_I: Picard
 * iteration of the implicit discrete-gradient scheme for (X, P, e_x), one
 * global e_x update per sweep; PIC_SUBSYSTEM_II: fixed point for
 * (e_y, e_z, a_y, a_z) with the exact solve of (M0 + dt^2/4 G^T M1 G);
 * PIC_SUBSYSTEM_III (hbar != 0): every spin rotated by the exact Rodrigues
 * formula (Eq. spin_rodrigue), r = (0, dA_z/dx, -dA_y/dx) at its marker.
 * With hbar != 0 subsystem I's momentum update carries the discrete gradient
 * of the Zeeman energy, -dt hbar (s_y D2_z - s_z D2_y) with D2 the path mean
 * of d^2A/dx^2, and subsystem II's right side the source
 * -dt hbar G^T Lambda_1(X)^T W S_z (y), +dt hbar G^T Lambda_1(X)^T W S_y (z).
 * *iters (may be NULL) receives the number of particle sweeps.
 * Starting fields: subsystem I starts from e_x^n; subsystem II from e_y^n,
 * e_z^n extrapolated in time by the polynomial through the states after the
 * handle's last (up to three) subsystem-II solves.  The fixed point does not
 * depend on the start, only the sweep count does.
 * PIC_ERR_NOCONVERGE when max_iter sweeps did not reach the tolerance (the
 * state is then the last iterate). */
int pic_substep(pic_handle *h, int32_t which, int32_t *iters);

/* nsteps steps: Lie--Trotter Phi_II(dt) o Phi_I(dt) (Sec. 5; with hbar != 0
 * Phi_III(dt) o Phi_II(dt) o Phi_I(dt)), or with
 * splitting = PIC_SPLIT_STRANG the symmetric Phi_I(dt/2) o Phi_II(dt) o
 * Phi_I(dt/2), each substep the paper's energy-conserving scheme.  Sweep counts
 * summed over the steps go to *iters_I / *iters_II (may be NULL). */
int pic_step(pic_handle *h, int32_t nsteps, int64_t *iters_I, int64_t *iters_II);

/* Discrete Hamiltonian (Eq. discrete_H) and Gauss-law residual, evaluated in
 * double from the stored state (out holds 7 doubles):
 *  out[0] = sum_a w (gamma(p_a, A_h(x_a)) - 1)     kinetic
 *  out[1] = 1/2 e_x^T M1 e_x
 *  out[2] = 1/2 (e_y^T M0 e_y + e_z^T M0 e_z)
 *  out[3] = 1/2 (a_y^T K a_y + a_z^T K a_z),  K = G^T M1 G
 *  out[4] = total = out[0]+out[1]+out[2]+out[3]+out[6]
 *  out[5] = max_j |(G^T M1 e_x)_j + rho_j - dx|   (discrete Poisson residual)
 *  out[6] = hbar sum_a w (s_y dA_z/dx - s_z dA_y/dx)(x_a)   Zeeman (0 without spin) */
int pic_energy(pic_handle *h, double out[7]);

/* Kernel timing of the hot loop (CUDA events on the handle's stream).
 * pic_timing_enable(h, 1) starts recording; pic_timing_read fills
 * out[0] = total ms in subsystem-I sweep kernels, out[1] = their launches,
 * out[2] = ms in subsystem-II sweep kernels, out[3] = launches,
 * out[4] = ms in grid solve kernels, out[5] = launches,
 * out[6] = total kernel launches issued by the library since enable,
 * out[7] = marker-sweeps done by subsystem-I sweep kernels (sum of N_p per launch),
 * out[8] = ms in warm-start network kernels, out[9] = their launches. */
int pic_timing_enable(pic_handle *h, int32_t on);
int pic_timing_read(pic_handle *h, double out[10]);

/* Release the handle and all memory it owns.  NULL is allowed. */
int pic_destroy(pic_handle *h);

/* ---------------------------------------------------------------------
 * Learned warm start of the subsystem-I fixed point.  The paper solves each
 * implicit substep by fixed-point iteration from x^(0) = x^n (Sec. 4.2); a
 * small network can propose x^(0) instead.  The iteration still runs to the
 * same tolerance, so the converged state does not depend on the proposal.
 * Network: 6 inputs (cell-relative x, p, E_x(x^n), A_y(x^n), A_z(x^n), dt),
 * normalised by (v - shift) * scale; three hidden layers of width 64, GELU
 * (tanh form); 2 outputs times out_scale, read as
 *   y0 = (x^{n+1} - x^n - dt p / gamma(p, A(x^n))) / dt^2,
 *   y1 = (p^{n+1} - p^n - dt E_x(x^n)) / dt^2.
 * Parameters: 8898 floats, W1 (64x6 row-major [out][in]), b1, W2 (64x64), b2,
 * W3, b3, W4 (2x64), b4.  norm: 14 floats, shift[6], scale[6], out_scale[2].
 * Inference: bf16 tensor cores with fp32 accumulation; training: fp32.
 * All X / T / Y / grad arrays are device pointers, row-major per sample.
 * --------------------------------------------------------------------- */
typedef struct pic_mlp pic_mlp;

/* Create a network on the current device.  params: 8898 host floats or NULL
 * (zeros); norm: 14 host floats (required). */
int pic_mlp_create(const float *params, const float *norm, void *stream, pic_mlp **out);
int pic_mlp_destroy(pic_mlp *m);
/* Copy the current fp32 parameters to host memory (8898 floats). */
int pic_mlp_get_params(pic_mlp *m, float *params_host);
/* Loss and its gradient on a batch: loss = mean_b sum_o (y_o - T_o / out_scale_o)^2
 * with y the normalised outputs of the fp32 network on X[B][6]; grad_out (device,
 * 8898 floats) and loss_out (host) may be NULL. */
int pic_mlp_grad(pic_mlp *m, const float *X, const float *T, int64_t B, float *grad_out, double *loss_out);
/* One Adam step (beta 0.9/0.999, eps 1e-8) on the batch loss above. */
int pic_mlp_train_step(pic_mlp *m, const float *X, const float *T, int64_t B, float lr, double *loss_out);
/* Y[B][2] = scaled outputs of the bf16 tensor-core network on raw features X[B][6]. */
int pic_mlp_infer(pic_mlp *m, const float *X, int64_t B, float *Y);
/* Attach a network to a handle created with warm_start = PIC_WARM_MLP (the
 * handle borrows it: keep it alive while the handle steps).  NULL detaches. */
int pic_set_warm_mlp(pic_handle *h, pic_mlp *m);

/* Message of the last error on h; with h == NULL, the message of the last
 * failed pic_init or pic_deposit_current_noalloc on the calling thread. */
const char *pic_last_error(const pic_handle *h);

/* Path-integrated current deposit for callers that cannot allocate device
 * memory (a memory pool that must not grow, a device heap owned by another
 * component, a plugin not allowed to hold CUDA allocations).  The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 * It needs no handle and calls no allocator; its scratch is a fixed 2 MiB
 * device array inside the library (one per GPU that loads the library, kept
 * until the process exits).
 *   out[nx] (device)  = sum_a weight * int_{x_a}^{x_a + disp_a} Lambda^1_i,
 * the same quantity as pic_deposit(PIC_DEP_CURRENT), computed in double.  Each
 * block sums its markers with shared-memory atomics (so repeated calls may
 * differ in the last bits) and the blocks' partial rows are then added in a
 * fixed order.  x[np], disp[np]: device arrays of positions (any finite value,
 * read periodically; normally in [0, L)) and signed displacements (length
 * units, at most 64 cells).  L > 0, 8 <= nx <= 8192 (larger grids exceed the
 * scratch and are rejected with PIC_ERR_INVALID), 2 <= degree <= 5 (degree of
 * V0; the deposit uses degree-1).  Work is ordered on `stream` (cudaStream_t
 * as void*); every call reads a status word back and synchronises that stream,
 * so it blocks the host until out is complete.  The first call on a device
 * (with that device current) sets up the scratch address and kernel attributes.
 * All calls share the one
 * scratch array, which keeps the last call's contents: calls whose kernels
 * overlap on the GPU (other streams or threads) race and give wrong results.
 * Errors: PIC_ERR_INVALID, PIC_ERR_NUMERIC (a position or displacement that is
 * not finite, or a displacement beyond 64 cells; out is then incomplete),
 * PIC_ERR_CUDA; message via pic_last_error(NULL). */
int pic_deposit_current_noalloc(double L, int32_t nx, int32_t degree, int64_t np, double weight,
                                const double *x, const double *disp, double *out, void *stream);

/* ---------------------------------------------------------------------
 * Batched ensembles.  Many independent runs of the method (each its own
 * configuration, grid and markers: Sec. 4.2 applied to each) advance together:
 * one step of the ensemble is one CUDA-graph launch in which every kernel
 * covers all runs.  Each run keeps its own fixed-point loops; the particle
 * sweeps are persistent kernels that take work items (a run and a range of its
 * markers) from a queue rebuilt before every sweep from the runs still
 * iterating, so a run that has converged drops out while the others go on.
 * The two loops are conditional (WHILE) graph nodes, ended on the device.
 * All runs must share degree, precision, warm start (PIC_WARM_NONE or
 * PIC_WARM_EXPLICIT) and warm_field (with warm_field = 1 each step first runs
 * the predicted start of every run: the proposals' currents over the work queue,
 * then e^(0) per run); grid size, marker count, weight, dt, tolerances and
 * sort interval may differ.  Runs use the default deposit accumulation,
 * Lie--Trotter steps and no spin.  1 <= nruns <= 1024.
 * --------------------------------------------------------------------- */
typedef struct pic_ensemble pic_ensemble;

/* Create the runs (as pic_init with cfgs[r], ins[r], mem) on `stream`.
 * use_graph = 1: steps run as one graph launch; 0: the same kernels with
 * the loops driven from the host (one readback per sweep), for checking.
 * Errors: PIC_ERR_INVALID (mixed degree / precision / warm start / warm_field,
 * an MLP warm start, another deposit accumulation, symmetric splitting, spin,
 * nruns out of range, or a run's own pic_init error), PIC_ERR_NOMEM,
 * PIC_ERR_CUDA; message via pic_last_error(NULL). */
int pic_ensemble_create(const pic_config *cfgs, const pic_arrays *ins, int32_t nruns, int32_t mem,
                        int32_t use_graph, void *stream, pic_ensemble **out);

/* Advance every run by nsteps steps (I then II, then each run's periodic
 * sort).  sweeps (host, may be NULL): 2*nruns counts, added to, of the
 * subsystem-I and -II sweeps of each run; status (host, may be NULL): nruns
 * values, 0 or PIC_ERR_NUMERIC / PIC_ERR_NOCONVERGE / PIC_ERR_CUDA (a bounded
 * wait gave up) per run; the bits stay set for the life of the ensemble.  A run
 * with PIC_ERR_NUMERIC or PIC_ERR_CUDA is stopped (keeps its state, takes no
 * more work); a run with PIC_ERR_NOCONVERGE goes on from its last iterate,
 * its loops capped at max_iter sweeps.  The other runs are not affected.
 * Returns the first failing run's error, or PIC_OK. */
int pic_ensemble_step(pic_ensemble *e, int32_t nsteps, int64_t *sweeps, int32_t *status);

/* Autotuner: pick the work-item size of the batched sweeps (markers per item)
 * and the number of persistent sweep blocks per SM by timing one ensemble step
 * per candidate (the steps are real steps: the runs advance) and keeping the
 * fastest per marker-sweep.  cache_path (may be NULL): a text file of earlier
 * choices keyed by device and ensemble shape; a hit skips the timing, a new
 * choice is appended.  choice (host, may be NULL): [markers per item, blocks
 * per SM, 1 if taken from the cache]. */
int pic_ensemble_tune(pic_ensemble *e, const char *cache_path, int32_t choice[3]);

/* Set the schedule by hand (markers per item: a positive multiple of 1024;
 * blocks per SM >= 1, at most what fits). */
int pic_ensemble_set_schedule(pic_ensemble *e, int32_t item_markers, int32_t blocks_per_sm);

/* The handle of run r (borrowed; valid until pic_ensemble_destroy): use it
 * with pic_energy, pic_get_state, pic_gather, pic_deposit. */
pic_handle *pic_ensemble_run(pic_ensemble *e, int32_t r);

/* Kernel launches issued by pic_ensemble_step since creation (graph nodes
 * executed, counted from the device's loop counters). */
int64_t pic_ensemble_launches(const pic_ensemble *e);

int pic_ensemble_destroy(pic_ensemble *e);
const char *pic_ensemble_last_error(const pic_ensemble *e);

/* Library version string, e.g. "libpic 1.0 sm_103a". */
const char *pic_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H_ */
