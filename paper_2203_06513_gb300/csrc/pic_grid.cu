// pic_grid.cu -- grid-side kernels of libpic (double precision) and the host
// algebra of the periodic spline matrices.
//
// Every matrix of the method is a symmetric circulant on M nodes (Sec. 3.1):
//   M0 (degree k), M1 (degree k-1), K = G^T M1 G, P = M0 + dt^2/4 K.
// Solves apply the exact inverse as a circulant convolution: the inverse of a
// banded SPD circulant has a first row that decays geometrically, so it is
// truncated where its entries fall below 1e-17 of the largest (or kept whole).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "pic_internal.h"

namespace pic {

// ---------------------------------------------------------------------------
// Host: exact mass-matrix bands.  (M_d)_{0,r} = int N^d(s) N^d(s - r) ds * dx,
// the autocorrelation of the cardinal B-spline, equals dx N^{2d+1}(d + 1 + r).
// N^n is evaluated from the truncated-power form
//   N^n(s) = 1/n! sum_{i=0}^{n+1} (-1)^i C(n+1, i) (s - i)_+^n,
// exact in rational arithmetic; at the integer arguments used here every term
// is an integer divided by n!, so double evaluation is exact for n <= 11.
// ---------------------------------------------------------------------------
static double cardinal_tp(int n, double s)
{
    double acc = 0.0, binom = 1.0, fact = 1.0;
    for (int i = 1; i <= n; ++i) fact *= i;
    for (int i = 0; i <= n + 1; ++i) {
        const double u = s - i;
        if (u > 0.0) acc += ((i & 1) ? -1.0 : 1.0) * binom * std::pow(u, n);
        binom = binom * (n + 1 - i) / (i + 1);
    }
    return acc / fact;
}

int mean_scale(int d)
{
    static const int S[] = {1, 1, 6, 6, 120};
    return (d >= 0 && d <= 4) ? S[d] : 0;
}

void mass_band(int d, double dx, double *band)
{
    for (int r = 0; r <= d; ++r) band[r] = dx * cardinal_tp(2 * d + 1, (double)(d + 1 + r));
}

// First row g of the inverse of the symmetric circulant with band c_0..c_bw:
// eigenvalues lambda_m = c_0 + 2 sum_d c_d cos(2 pi m d / M), g_d = 1/M sum_m
// cos(2 pi m d / M) / lambda_m, with one step of iterative refinement.  The
// cosine table is made exactly symmetric (cs[M - j] = cs[j]), so both transforms
// are symmetric in their output index bit for bit and only the first half is
// summed; indices m q mod M advance by addition.
static void inverse_taps_compute(const double *band, int bw, int M, double cut, double *g, int *d_start,
                                 int *ntap, double *taps)
{
    const double twopi = 6.283185307179586476925286766559;
    std::vector<double> cs(M), lam(M), r(M), corr(M);
    for (int m = 0; m <= M / 2; ++m) cs[m] = std::cos(twopi * (double)m / (double)M);
    for (int m = M / 2 + 1; m < M; ++m) cs[m] = cs[M - m];
    for (int m = 0; m < M; ++m) {
        double l = band[0];
        for (int d = 1; d <= bw; ++d) l += 2.0 * band[d] * cs[(long long)m * d % M];
        lam[m] = 1.0 / l;
    }
    // y_k = sum_j v_j cs[k j mod M] for k = 0 .. M/2, mirrored; four interleaved
    // compensated partial sums (independent chains), added at the end
    auto cos_transform = [&](const std::vector<double> &v, std::vector<double> &y) {
        for (int k = 0; k <= M / 2; ++k) {
            double s[4] = {0.0, 0.0, 0.0, 0.0}, comp[4] = {0.0, 0.0, 0.0, 0.0};
            int idx = 0;
            for (int j = 0; j < M; ++j) {
                const int l = j & 3;
                const double t = v[j] * cs[idx] - comp[l];
                const double tt = s[l] + t;
                comp[l] = (tt - s[l]) - t;
                s[l] = tt;
                idx += k;
                if (idx >= M) idx -= M;
            }
            y[k] = ((s[0] + s[1]) + (s[2] + s[3])) - ((comp[0] + comp[1]) + (comp[2] + comp[3]));
        }
        for (int k = M / 2 + 1; k < M; ++k) y[k] = y[M - k];
    };
    auto apply_inv = [&](const std::vector<double> &rhs_even, std::vector<double> &out) {
        // rhs is symmetric (even) so its DFT is real: R_m = sum_q rhs_q cos(2 pi m q / M)
        std::vector<double> R(M);
        cos_transform(rhs_even, R);
        for (int m = 0; m < M; ++m) R[m] *= lam[m];
        cos_transform(R, out);
        for (int d = 0; d < M; ++d) out[d] /= (double)M;
    };
    std::vector<double> e0(M, 0.0), gv(M);
    e0[0] = 1.0;
    apply_inv(e0, gv);
    // refinement: r = e0 - A g, g += A^{-1} r
    for (int i = 0; i < M; ++i) {
        double s = band[0] * gv[i];
        for (int d = 1; d <= bw; ++d) s += band[d] * (gv[(i + d) % M] + gv[(i - d + M) % M]);
        r[i] = e0[i] - s;
    }
    apply_inv(r, corr);
    for (int i = 0; i < M; ++i) gv[i] += corr[i];
    for (int i = 0; i < M; ++i) g[i] = gv[i];
    double gmax = 0.0;
    for (int i = 0; i < M; ++i) gmax = std::fmax(gmax, std::fabs(gv[i]));
    int T = 0;
    for (int d = 1; d <= M / 2; ++d)
        if (std::fabs(gv[d]) > cut * gmax) T = d;
    if (2 * T + 1 <= M && !(M % 2 == 0 && T == M / 2)) {
        *d_start = -T;
        *ntap = 2 * T + 1;
        for (int n = 0; n < 2 * T + 1; ++n) taps[n] = gv[(n - T + M) % M];
    } else {  // whole circulant: offsets -(M/2 - 1) .. M/2 (M entries)
        const int lo = -(M / 2 - 1 + (M % 2));
        *d_start = lo;
        *ntap = M;
        for (int n = 0; n < M; ++n) taps[n] = gv[((lo + n) % M + M) % M];
    }
}

// The taps of one (band, M, cut) are the same for every handle that asks: a
// process-wide table of the recent ones spares repeated set-ups the O(M^2) work.
void inverse_taps(const double *band, int bw, int M, double cut, double *g, int *d_start, int *ntap,
                  double *taps)
{
    struct Entry {
        std::vector<double> key, g, taps;
        int d_start, ntap;
    };
    static std::mutex mu;
    static std::vector<Entry> table;
    std::vector<double> key(band, band + bw + 1);
    key.push_back((double)M);
    key.push_back(cut);
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : table)
            if (e.key == key) {
                std::copy(e.g.begin(), e.g.end(), g);
                std::copy(e.taps.begin(), e.taps.end(), taps);
                *d_start = e.d_start;
                *ntap = e.ntap;
                return;
            }
    }
    inverse_taps_compute(band, bw, M, cut, g, d_start, ntap, taps);
    std::lock_guard<std::mutex> lock(mu);
    if (table.size() >= 64) table.clear();
    table.push_back(Entry{key, std::vector<double>(g, g + M), std::vector<double>(taps, taps + *ntap), *d_start,
                          *ntap});
}

// ---------------------------------------------------------------------------
// Convergence decision, made by the last block of a solve kernel.
// FP64 form (Sec. 5, tolerance tol): max |x^(k+1) - x^(k)| <= tol (length) and
// max |e^(k+1) - e^(k)| <= tol.  FP32 form: position increments at the float
// resolution of the offset (dtol, relative to max(1, |delta|)) and field
// increments below tol or no longer shrinking (stagnation at float noise).
// ---------------------------------------------------------------------------
__device__ void decide(const ConvArgs &A)
{
    DevCtrl *c = A.ctrl;
    __threadfence();
    if (A.count) *A.count += 1;
    const double d = (A.subsystem == 1) ? bits_to_double(c->dmax_bits) : 0.0;
    const double e = bits_to_double(c->emax_bits);
    const double ep = bits_to_double(c->eprev_bits);
    c->iter += 1;
    bool ok;
    if (!A.fp32) {
        ok = (d * A.dx <= A.tol) && (e <= A.tol);
    } else {
        // Float iterates stop improving at rounding noise, so increments alone never
        // reach a tight tolerance.  Estimate the remaining error of the new iterate
        // from the increment v_k and the observed contraction r = v_k / v_{k-1}
        // (geometric tail v_k r / (1 - r), r capped at 0.9), and stop when both the
        // position and field estimates are below tolerance, or when both increments
        // have stopped shrinking at noise level.
        const double dp = bits_to_double(c->dprev_bits);
        auto est = [](double v, double vprev) {
            if (v == 0.0) return 0.0;
            // no previous increment (first sweep): no contraction estimate yet
            double r = (vprev < 1e300) ? v / vprev : 0.9;
            if (!(r < 0.9)) r = 0.9;
            return v * r / (1.0 - r);
        };
        // field tolerance.  Subsystem I: the absolute tol, or erel of the field's
        // max-norm when that is larger, on the last increment itself: the markers'
        // momenta were updated with the field of the sweep before, and that
        // mismatch is proportional to the last increment (not to the estimated
        // remaining error), with a sign that does not average out over steps: a
        // rule on the estimate accepted increments near 1e-7 of the field and let
        // the energy drift by 1e-12 of the total a step on C2.
        // Subsystem II: the estimated remaining error below the absolute tol.  Its
        // markers do not move, the sweep is deterministic, and the remaining field
        // error enters the transverse energy directly.
        const double emag = bits_to_double(c->emag_bits);
        const bool dok = (A.subsystem == 1) ? (est(d, dp) <= A.dtol) : true;
        const bool eok = (A.subsystem == 1) ? (e <= fmax(A.tol, A.erel * emag)) : (est(e, ep) <= A.tol);
        const bool dstag = (A.subsystem == 1) ? (d >= 0.5 * dp && d <= 1e-4) : true;
        const bool estag = e >= 0.5 * ep && e <= 1e-8;
        ok = (dok && eok) || (c->iter >= 3 && dstag && estag);
    }
    bool stop = ok;
    if (!ok && c->iter >= A.max_iter) {
        c->status |= STATUS_NOCONV;
        stop = true;
    }
    if (c->status & (STATUS_NUMERIC | STATUS_TIMEOUT)) stop = true;
    c->converged = stop ? 1 : 0;
    c->dprev_bits = c->dmax_bits;
    c->eprev_bits = c->emax_bits;
    c->dmax_bits = 0ull;
    c->emax_bits = 0ull;
    c->emag_bits = 0ull;
    c->ticket = 0u;
    __threadfence();
    if (A.graph && A.cond_handle)
        cudaGraphSetConditional((cudaGraphConditionalHandle)A.cond_handle, stop ? 0u : 1u);
}

// float images of sweep I: a / K! rounded, their differences, ebar dx / S1 rounded
__device__ __forceinline__ void image1_at(int i, int M, const double *ay, const double *az, double ebar,
                                          const StageImages &img)
{
    const int im = (i == 0) ? M - 1 : i - 1;
    const float y = (float)(ay[i] * img.inv_fact), ym = (float)(ay[im] * img.inv_fact);
    const float z = (float)(az[i] * img.inv_fact), zm = (float)(az[im] * img.inv_fact);
    img.a[i] = make_float2(y, z);
    img.f[i] = make_float4((float)(ebar * img.escale), y - ym, z - zm, 0.f);
}

// float images of sweep II for one component c: a^(k) / K! rounded and the residue
// of the sum a^n / K! + a^(k) / K! after both roundings
__device__ __forceinline__ void image2_at(int i, int c, double an, double ak, const StageImages &img)
{
    const double n = an * img.inv_fact, k = ak * img.inv_fact;
    const float hn = (float)n, hk = (float)k;
    const float lo = (float)((n - (double)hn) + (k - (double)hk));
    float *pk = reinterpret_cast<float *>(&img.ak[i]), *pl = reinterpret_cast<float *>(&img.lo[i]);
    pk[c] = hk;
    pl[c] = lo;
}

// y_i = sum_n taps[n] in[(i - (d_start + n)) mod M], one output per thread,
// input and taps staged in shared memory (input twice, so no index wraps).
// Block bx of component comp; returns true in the one block that finished the
// run's solve last (after the convergence decision, in the solve modes).
__device__ bool conv_block(const ConvArgs &A, int bx, int comp, double *s_conv, double *s_red)
{
    const int M = A.M;
    double *s_in = s_conv;              // 2M
    double *s_tap = s_conv + 2 * M;     // ntap
    const double *in = A.in[comp];
    double *zero = A.zero[comp];
    if (A.graph && A.mode != CONV_PLAIN) {   // replayed by a graph: buffers by sweep parity
        const int it = *reinterpret_cast<volatile const int *>(&A.ctrl->iter);
        in = A.pair[comp][it & 1];
        zero = A.pair[comp][(it + 1) & 1];
    }
    const int off = M / 2;              // s_in[q] = in[(q - off) mod M], q in [0, 2M)
    for (int q = threadIdx.x; q < 2 * M; q += blockDim.x) {
        int g = q - off;
        g = g < 0 ? g + M : (g >= M ? g - M : g);
        s_in[q] = in[g];
    }
    for (int n = threadIdx.x; n < A.ntap; n += blockDim.x) s_tap[n] = A.taps[n];
    __syncthreads();
    const int i = bx * blockDim.x + threadIdx.x;
    double diff = 0.0, mag = 0.0;
    if (i < M) {
        // offsets d = d_start + n lie in [-(M-1)/2, M/2], so i - d + off is in [0, 2M)
        const double *base = s_in + (i - A.d_start + off);
        double acc0 = 0.0, acc1 = 0.0;
        int n = 0;
        for (; n + 1 < A.ntap; n += 2) {
            acc0 = fma(s_tap[n], base[-n], acc0);
            acc1 = fma(s_tap[n + 1], base[-n - 1], acc1);
        }
        if (n < A.ntap) acc0 = fma(s_tap[n], base[-n], acc0);
        const double y = acc0 + acc1;
        if (A.mode == CONV_PLAIN) {
            A.out[comp][i] = y;
        } else if (A.mode == CONV_START1) {
            const double en = A.en[0][i];
            const double e0 = en - y;                    // e^(0) = e^n - M1^{-1} j^(0)
            A.ek[0][i] = e0;
            A.aux[0][i] = 0.5 * (en + e0);
            if (A.img.f) reinterpret_cast<float *>(A.img.f)[4 * i] = (float)(0.5 * (en + e0) * A.img.escale);
        } else if (A.mode == CONV_SOLVE1) {
            const double en = A.en[0][i];
            const double enew = en - y;                  // e^(k+1) = e^n - M1^{-1} j
            diff = fabs(enew - A.ek[0][i]);
            mag = fabs(enew);
            A.ek[0][i] = enew;
            A.aux[0][i] = 0.5 * (en + enew);             // ebar for the next sweep
            if (A.img.f) reinterpret_cast<float *>(A.img.f)[4 * i] = (float)(0.5 * (en + enew) * A.img.escale);
            zero[i] = 0.0;
        } else {                                         // CONV_SOLVE2
            const double en = A.en[comp][i];
            const double enew = A.r0[comp][i] + A.dt * y;   // P e^(k+1) = b + dt s
            diff = fabs(enew - A.ek[comp][i]);
            mag = fabs(enew);
            A.ek[comp][i] = enew;
            const double ak = A.an[comp][i] - 0.5 * A.dt * (en + enew);   // a^(k+1)
            A.aux[comp][i] = ak;
            if (A.img.ak) image2_at(i, comp, A.an[comp][i], ak, A.img);
            zero[i] = 0.0;
        }
    }
    if (A.mode == CONV_PLAIN || A.mode == CONV_START1) return false;
    block_max_to(&A.ctrl->emax_bits, diff, s_red);
    block_max_to(&A.ctrl->emag_bits, mag, s_red);
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int nblk = (unsigned)(((M + blockDim.x - 1) / blockDim.x) * A.ncomp);
        const unsigned int t = atomicAdd(&A.ctrl->ticket, 1u);
        s_last = (t == nblk - 1) ? 1 : 0;
        if (s_last) decide(A);
    }
    __syncthreads();
    return s_last != 0;
}

__global__ void __launch_bounds__(64) k_conv(ConvArgs A)
{
    extern __shared__ __align__(16) double s_conv[];
    __shared__ double s_red[32];
    conv_block(A, blockIdx.x, blockIdx.y, s_conv, s_red);
}

// Batched solves of an ensemble: block (bx, run, comp).  Runs that are not in
// the current sweep (converged, or stopped by an error) are skipped.  After a
// run's decision, the last run to decide in this sweep records whether any run
// goes on, and sets the loop's conditional handle (graph mode).
__global__ void __launch_bounds__(64) k_conv_ens(const ConvArgs *runs, EnsQueue *Q, int *sweeps,
                                                 unsigned long long cond)
{
    extern __shared__ __align__(16) double s_conv[];
    __shared__ double s_red[32];
    const int r = blockIdx.y, comp = blockIdx.z;
    const ConvArgs &A = runs[r];
    if (A.mode != CONV_PLAIN && !Q->active[r]) return;
    if (comp >= A.ncomp || (int)(blockIdx.x * blockDim.x) >= A.M) return;
    const bool last = conv_block(A, blockIdx.x, comp, s_conv, s_red);
    if (!last || threadIdx.x != 0) return;
    atomicAdd(&sweeps[2 * r + A.subsystem - 1], 1);
    if (!A.ctrl->converged) atomicAdd(&Q->n_continue, 1);
    __threadfence();
    const int t = atomicAdd(&Q->n_decided, 1);
    if (t == Q->nactive - 1) {
        __threadfence();
        const int go = atomicAdd(&Q->n_continue, 0) > 0 ? 1 : 0;
        Q->go = go;
        Q->loops[A.subsystem - 1] += 1;
        if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, (unsigned)go);
    }
}

static int conv_optin(const void *fn, size_t smem, size_t &opted)
{
    if (smem > 48 * 1024 && smem > opted) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return 1;
        opted = smem;
    }
    return 0;
}

static size_t g_conv_ens_opted = 0;

// raise the shared-memory limit of k_conv_ens before any capture of it
int conv_ens_optin(int Mmax, int ntap_max)
{
    const size_t smem = (2 * (size_t)Mmax + (size_t)ntap_max) * sizeof(double);
    return conv_optin((const void *)k_conv_ens, smem, g_conv_ens_opted);
}

int launch_conv_ens(const ConvArgs *runs, int nruns, int Mmax, int ncomp, int ntap_max, EnsQueue *Q,
                    int *sweeps, unsigned long long cond, cudaStream_t s)
{
    const size_t smem = (2 * (size_t)Mmax + (size_t)ntap_max) * sizeof(double);
    if (smem > 48 * 1024 && smem > g_conv_ens_opted) return 1;   // conv_ens_optin first
    dim3 grid((Mmax + 63) / 64, nruns, ncomp);
    k_conv_ens<<<grid, 64, smem, s>>>(runs, Q, sweeps, cond);
    return 0;
}

int launch_conv(const ConvArgs &a, cudaStream_t s)
{
    const int threads = 64;
    dim3 grid((a.M + threads - 1) / threads, a.ncomp);
    const size_t smem = (2 * (size_t)a.M + (size_t)a.ntap) * sizeof(double);
    static size_t opted = 0;   // largest dynamic shared memory opted in so far
    if (conv_optin((const void *)k_conv, smem, opted)) return 1;
    k_conv<<<grid, threads, smem, s>>>(a);
    return 0;
}

// Control block at the start of a fixed-point loop (the error bits and the field
// history counts stay).
__device__ __forceinline__ void ctrl_loop_reset(DevCtrl *ctrl)
{
    ctrl->dmax_bits = 0ull;
    ctrl->emax_bits = 0ull;
    ctrl->emag_bits = 0ull;
    ctrl->dprev_bits = 0x7ff0000000000000ull;
    ctrl->eprev_bits = 0x7ff0000000000000ull;
    ctrl->iter = 0;
    ctrl->converged = 0;
    ctrl->ticket = 0u;
}

// Starting field of a fixed-point iteration.  The fixed point does not depend on
// it, only the number of sweeps to reach it does: e^n extrapolated in time by the
// polynomial through the last q + 1 states, q = min(stored changes, order):
// e^n, e^n + d0, e^n + 2 d0 - d1, e^n + 3 d0 - 3 d1 + d2.
__device__ __forceinline__ double start_field(double e, double *const d[kMaxStartOrder], int i, int q)
{
    switch (q) {
    case 0: return e;
    case 1: return e + d[0][i];
    case 2: return e + (2.0 * d[0][i] - d[1][i]);
    default: return e + (3.0 * (d[0][i] - d[1][i]) + d[2][i]);
    }
}

// ---------------------------------------------------------------------------
// Subsystem I preparation: e^(0), ebar^(0) = (e^n + e^(0)) / 2, the gradients
// (G a)_i = (a_i - a_{i-1}) / dx, cleared deposits, the float images, the
// control block reset for the loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prep1_at(int i, const RunDesc &R)
{
    const int M = R.M;
    const int q = min(R.ctrl->hist1, R.fh.order1);    // hist1: written only by the commit kernel
    if (i < M) {
        const double e0 = start_field(R.ex[i], R.fh.x, i, q);
        const double eb = 0.5 * (R.ex[i] + e0);
        if (R.img.a) image1_at(i, M, R.ay, R.az, eb, R.img);
        const int im = (i == 0) ? M - 1 : i - 1;
        R.ga_y[i] = (R.ay[i] - R.ay[im]) / R.dx;
        R.ga_z[i] = (R.az[i] - R.az[im]) / R.dx;
        R.ek[i] = e0;
        R.ebar[i] = eb;
        R.j0[i] = 0.0;
        R.j1[i] = 0.0;
    }
    if (i == 0) ctrl_loop_reset(R.ctrl);
}

__global__ void k_prep1(RunDesc R) { prep1_at(blockIdx.x * blockDim.x + threadIdx.x, R); }

__global__ void k_prep1_ens(const RunDesc *runs)
{
    prep1_at(blockIdx.x * blockDim.x + threadIdx.x, runs[blockIdx.y]);
}

int launch_prep1_ens(const RunDesc *R, int nruns, int Mmax, cudaStream_t s)
{
    k_prep1_ens<<<dim3((Mmax + 255) / 256, nruns), 256, 0, s>>>(R);
    return 0;
}

int launch_prep1(const RunDesc &R, cudaStream_t s)
{
    k_prep1<<<(R.M + 255) / 256, 256, 0, s>>>(R);
    return 0;
}

// ---------------------------------------------------------------------------
// Subsystem II preparation: b = (M0 - dt^2/4 K) e^n + dt K a^n (banded
// circulant products), e^(0), a^(0) = a^n - dt/2 (e^n + e^(0)), cleared
// deposits, the float images, the control block reset for the loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prep2_at(int i, const RunDesc &R)
{
    const int M = R.M, K = R.K;
    const double dt = R.dt;
    const int q = min(R.ctrl->hist2, R.fh.order2);    // hist2: written only by the commit kernel
    if (i < M) {
        const double *ey = R.ey, *ez = R.ez, *ay = R.ay, *az = R.az;
        const double ey0 = start_field(ey[i], R.fh.y, i, q);
        const double ez0 = start_field(ez[i], R.fh.z, i, q);
        const double ay0 = ay[i] - 0.5 * dt * (ey[i] + ey0), az0 = az[i] - 0.5 * dt * (ez[i] + ez0);
        if (R.img.an) {
            R.img.an[i] = make_float2((float)(ay[i] * R.img.inv_fact), (float)(az[i] * R.img.inv_fact));
            image2_at(i, 0, ay[i], ay0, R.img);
            image2_at(i, 1, az[i], az0, R.img);
        }
        double vy = R.rowPm[0] * ey[i] + dt * R.rowK[0] * ay[i];
        double vz = R.rowPm[0] * ez[i] + dt * R.rowK[0] * az[i];
        for (int d = 1; d <= K; ++d) {
            const int ip = (i + d) % M, im = (i - d + M) % M;
            vy += R.rowPm[d] * (ey[ip] + ey[im]) + dt * R.rowK[d] * (ay[ip] + ay[im]);
            vz += R.rowPm[d] * (ez[ip] + ez[im]) + dt * R.rowK[d] * (az[ip] + az[im]);
        }
        R.by[i] = vy;
        R.bz[i] = vz;
        R.eky[i] = ey0;
        R.ekz[i] = ez0;
        R.aky[i] = ay0;
        R.akz[i] = az0;
        R.sy0[i] = 0.0; R.sz0[i] = 0.0; R.sy1[i] = 0.0; R.sz1[i] = 0.0;
    }
    if (i == 0) ctrl_loop_reset(R.ctrl);
}

__global__ void k_prep2(RunDesc R) { prep2_at(blockIdx.x * blockDim.x + threadIdx.x, R); }

__global__ void k_prep2_ens(const RunDesc *runs)
{
    prep2_at(blockIdx.x * blockDim.x + threadIdx.x, runs[blockIdx.y]);
}

int launch_prep2_ens(const RunDesc *R, int nruns, int Mmax, cudaStream_t s)
{
    k_prep2_ens<<<dim3((Mmax + 255) / 256, nruns), 256, 0, s>>>(R);
    return 0;
}

int launch_prep2(const RunDesc &R, cudaStream_t s)
{
    k_prep2<<<(R.M + 255) / 256, 256, 0, s>>>(R);
    return 0;
}

// e^{n+1} = e^(k) replaces e^n; its change enters the history (d[2] = d[1],
// d[1] = d[0], d[0] = e^{n+1} - e^n), as deep as the extrapolation order needs.
__device__ __forceinline__ void commit_field(int i, const double *ek, double *e, double *const d[kMaxStartOrder],
                                             int order)
{
    const double v = ek[i];
    for (int m = order - 1; m > 0; --m) d[m][i] = d[m - 1][i];
    if (order > 0) d[0][i] = v - e[i];
    e[i] = v;
}

// End of a substep: I: e_x = e^(k); II: e_perp = e^(k), a_perp = a^(k).  Thread
// 0 counts the stored changes (up to kMaxStartOrder) for the next preparation.
__device__ __forceinline__ void commit_at(int i, const RunDesc &R, int which)
{
    if (i < R.M) {
        if (which == 1) {
            commit_field(i, R.ek, R.ex, R.fh.x, R.fh.order1);
        } else {
            commit_field(i, R.eky, R.ey, R.fh.y, R.fh.order2);
            commit_field(i, R.ekz, R.ez, R.fh.z, R.fh.order2);
            R.ay[i] = R.aky[i];
            R.az[i] = R.akz[i];
        }
    }
    if (i == 0) {
        int *h = which == 1 ? &R.ctrl->hist1 : &R.ctrl->hist2;
        if (*h < kMaxStartOrder) *h += 1;
    }
}

__global__ void k_commit(RunDesc R, int which) { commit_at(blockIdx.x * blockDim.x + threadIdx.x, R, which); }

int launch_commit(const RunDesc &R, int which, cudaStream_t s)
{
    k_commit<<<(R.M + 255) / 256, 256, 0, s>>>(R, which);
    return 0;
}

// The same for every run of an ensemble.  Runs stopped by an error keep their
// fields and history.
__global__ void k_commit_ens(const RunDesc *runs, int which)
{
    const RunDesc &R = runs[blockIdx.y];
    if (R.ctrl->status & (STATUS_NUMERIC | STATUS_TIMEOUT)) return;
    commit_at(blockIdx.x * blockDim.x + threadIdx.x, R, which);
}

int launch_commit_ens(const RunDesc *R, int nruns, int Mmax, int which, cudaStream_t s)
{
    k_commit_ens<<<dim3((Mmax + 255) / 256, nruns), 256, 0, s>>>(R, which);
    return 0;
}

// Work list of the next batched sweep: the runs still iterating (not converged,
// not stopped by an error), each cut into items of item_markers markers;
// item_start is the exclusive prefix sum of the items per run.
__global__ void __launch_bounds__(1024) k_ens_plan(EnsQueue *Q, const EnsRun *runs, int nruns,
                                                   unsigned long long cond)
{
    __shared__ int s_scan[1024];
    __shared__ int s_nact[32];
    const int r = threadIdx.x;
    int items = 0, act = 0;
    if (r < nruns) {
        const DevCtrl *c = runs[r].ctrl;
        act = (!c->converged && !(c->status & (STATUS_NUMERIC | STATUS_TIMEOUT))) ? 1 : 0;
        const long long im = Q->item_markers;
        items = act ? (int)((runs[r].np + im - 1) / im) : 0;
        Q->active[r] = act;
    }
    // inclusive scan (Hillis-Steele) over the block
    s_scan[r] = items;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = r >= o ? s_scan[r - o] : 0;
        __syncthreads();
        s_scan[r] += v;
        __syncthreads();
    }
    if (r < nruns) Q->item_start[r + 1] = s_scan[r];
    const unsigned b = __ballot_sync(0xffffffffu, act != 0);
    if ((r & 31) == 0) s_nact[r >> 5] = __popc(b);
    __syncthreads();
    if (r == 0) {
        int n = 0;
        for (int w = 0; w < 32; ++w) n += s_nact[w];
        Q->item_start[0] = 0;
        Q->nitems = s_scan[nruns - 1];
        Q->nactive = n;
        Q->next = 0;
        Q->n_decided = 0;
        Q->n_continue = 0;
        Q->go = 0;
        // no run left (every run stopped by an error): no solve will decide, so the
        // loop is ended here
        if (n == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    }
}

__global__ void k_ens_status(const EnsRun *runs, int nruns, int *status)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nruns) status[r] = runs[r].ctrl->status;
}

int launch_ens_status(const EnsRun *runs, int nruns, int *status, cudaStream_t s)
{
    k_ens_status<<<(nruns + 255) / 256, 256, 0, s>>>(runs, nruns, status);
    return 0;
}

int launch_ens_plan(EnsQueue *Q, const EnsRun *runs, int nruns, unsigned long long cond, cudaStream_t s)
{
    if (nruns < 1 || nruns > kEnsMaxRuns) return 1;
    k_ens_plan<<<1, 1024, 0, s>>>(Q, runs, nruns, cond);
    return 0;
}

// Discrete Poisson right side: with r = -rho + dx, d = M1 e_x solves
// (d_j - d_{j+1}) / dx = r_j (Remark 2, Sec. 4.2): a running sum made mean-free.
__global__ void k_poisson_rhs(int M, double dx, const double *rho, double *d)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double run = 0.0, sum = 0.0;
    for (int j = 0; j < M; ++j) {
        d[j] = run;
        sum += run;
        run -= dx * (dx - rho[j]);
    }
    const double mean = sum / M;
    for (int j = 0; j < M; ++j) d[j] -= mean;
}

int launch_poisson_rhs(int M, double dx, const double *rho, double *d, cudaStream_t s)
{
    k_poisson_rhs<<<1, 32, 0, s>>>(M, dx, rho, d);
    return 0;
}

// Field energies (Eq. discrete_H) and the Gauss-law residual (Remark 2, Sec. 4.2).
__global__ void k_energy_grid(int M, int K, double dx, const double *rowM0, const double *rowM1,
                              const double *rowK, const double *ex, const double *ey,
                              const double *ez, const double *ay, const double *az,
                              const double *rho, double *diag)
{
    __shared__ double s_red[32];
    double eex = 0.0, eperp = 0.0, aperp = 0.0, gres = 0.0;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double m1e = rowM1[0] * ex[i], m1e_next = 0.0;
        const int inx = (i + 1) % M;
        m1e_next = rowM1[0] * ex[inx];
        for (int d = 1; d <= K - 1; ++d) {
            m1e += rowM1[d] * (ex[(i + d) % M] + ex[(i - d + M) % M]);
            m1e_next += rowM1[d] * (ex[(inx + d) % M] + ex[(inx - d + M) % M]);
        }
        double m0y = rowM0[0] * ey[i], m0z = rowM0[0] * ez[i];
        double ky = rowK[0] * ay[i], kz = rowK[0] * az[i];
        for (int d = 1; d <= K; ++d) {
            const int ip = (i + d) % M, im = (i - d + M) % M;
            m0y += rowM0[d] * (ey[ip] + ey[im]);
            m0z += rowM0[d] * (ez[ip] + ez[im]);
            ky += rowK[d] * (ay[ip] + ay[im]);
            kz += rowK[d] * (az[ip] + az[im]);
        }
        eex += 0.5 * ex[i] * m1e;
        eperp += 0.5 * (ey[i] * m0y + ez[i] * m0z);
        aperp += 0.5 * (ay[i] * ky + az[i] * kz);
        const double r = (m1e - m1e_next) / dx + rho[i] - dx;
        gres = fmax(gres, fabs(r));
    }
    double v;
    v = warp_sum(eex);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) { double s = 0; for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w]; diag[1] = s; }
    __syncthreads();
    v = warp_sum(eperp);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) { double s = 0; for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w]; diag[2] = s; }
    __syncthreads();
    v = warp_sum(aperp);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) { double s = 0; for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w]; diag[3] = s; }
    __syncthreads();
    v = warp_max(gres);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) { double s = 0; for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, s_red[w]); diag[5] = s; }
}

int launch_energy_grid(int M, int K, double dx, const double *rowM0, const double *rowM1,
                       const double *rowK, const double *ex, const double *ey, const double *ez,
                       const double *ay, const double *az, const double *rho, double *diag,
                       cudaStream_t s)
{
    k_energy_grid<<<1, 256, 0, s>>>(M, K, dx, rowM0, rowM1, rowK, ex, ey, ez, ay, az, rho, diag);
    return 0;
}

__global__ void k_ctrl_reset(DevCtrl *c)
{
    c->dmax_bits = 0ull;
    c->emax_bits = 0ull;
    c->emag_bits = 0ull;
    c->dprev_bits = 0x7ff0000000000000ull;
    c->eprev_bits = 0x7ff0000000000000ull;
    c->iter = 0;
    c->converged = 0;
    c->status = 0;
    c->ticket = 0u;
    c->hist1 = 0;
    c->hist2 = 0;
    c->acc[0] = c->acc[1] = c->acc[2] = c->acc[3] = 0.0;
}

int launch_ctrl_reset(DevCtrl *ctrl, cudaStream_t s)
{
    k_ctrl_reset<<<1, 1, 0, s>>>(ctrl);
    return 0;
}

}  // namespace pic

// Zeeman source of subsystem II (Sec. 4.2): b_y -= dt hbar (G^T d_z)_j and
// b_z += dt hbar (G^T d_y)_j, (G^T v)_j = (v_j - v_{j+1}) / dx, d = Lambda_1(X)^T W S.
__global__ void k_spin_rhs(int M, double dx, double c, const double *dy, const double *dz, double *by,
                           double *bz)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int jp = j + 1 == M ? 0 : j + 1;
    by[j] -= c * (dz[j] - dz[jp]) / dx;
    bz[j] += c * (dy[j] - dy[jp]) / dx;
}

namespace pic {
int launch_spin_rhs(int M, double dx, double dt, double hbar, const double *dy, const double *dz, double *by,
                    double *bz, cudaStream_t s)
{
    k_spin_rhs<<<(M + 255) / 256, 256, 0, s>>>(M, dx, dt * hbar, dy, dz, by, bz);
    return 0;
}
}  // namespace pic

// Split runs (markers over several processes): the marker-side results of a sweep
// that every process must agree on, packed as doubles for a max-reduction over
// processes: the largest position increment, and one entry per error bit (the max
// of 0/1 entries is their logical or).
__global__ void k_split_pack(const pic::DevCtrl *c, double *buf)
{
    buf[0] = pic::bits_to_double(c->dmax_bits);
    buf[1] = (c->status & pic::STATUS_NUMERIC) ? 1.0 : 0.0;
    buf[2] = (c->status & pic::STATUS_TIMEOUT) ? 1.0 : 0.0;
}

__global__ void k_split_unpack(pic::DevCtrl *c, const double *buf)
{
    c->dmax_bits = (unsigned long long)__double_as_longlong(buf[0]);
    if (buf[1] != 0.0) c->status |= pic::STATUS_NUMERIC;
    if (buf[2] != 0.0) c->status |= pic::STATUS_TIMEOUT;
}

namespace pic {
int launch_split_pack(const DevCtrl *c, double *buf, cudaStream_t s)
{
    k_split_pack<<<1, 1, 0, s>>>(c, buf);
    return 0;
}
int launch_split_unpack(DevCtrl *c, const double *buf, cudaStream_t s)
{
    k_split_unpack<<<1, 1, 0, s>>>(c, buf);
    return 0;
}
}  // namespace pic
