// pic_particles.cu -- marker kernels of libpic (sm_103a).
//
// Markers are stored as structure-of-arrays (cell int32, offset t, momentum p,
// iterates delta and p_new, caller index id) and kept sorted by the key
// (cell, velocity bin), so the 32 lanes of a warp hold markers of one or two
// cells with similar displacements.  Each sweep block owns one contiguous chunk
// of markers, reads it coalesced, stages the field coefficients once in shared
// memory (periodic halo of H cells, so no index wraps in the inner loop), and
// deposits through a per-warp register window (DepWindow) into a double row in
// shared memory, flushed to the global grid with one double atomic per node.
//
// Precision discipline of the FP32 form: per-marker arithmetic is float; the
// marker weight w and the cell width dx enter only when a window is flushed, in
// double; the momentum and position updates share one float factor
// tau = dt/dx (fields are staged as e dx and a_j - a_{j-1}), so the discrete
// work identity (p^(k+1) - p^n) vbar = (Ebar - F)(x^(k+1) - x^n) of Sec. 4.2
// holds with the same rounded factor on both sides.
#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

#include "pic_internal.h"

namespace pic {

template <typename R>
struct Real;
template <>
struct Real<float> { static constexpr bool fp32 = true; };
template <>
struct Real<double> { static constexpr bool fp32 = false; };

// Field tiles staged in shared memory, interleaved for vector loads.
template <typename R> struct FieldTile;
template <> struct FieldTile<float> {
    float2 *a;      // (a_y, a_z)
    float4 *f;      // (ebar dx, a_y,j - a_y,j-1, a_z,j - a_z,j-1, 0)
    __device__ __forceinline__ void aa(int i, float &y, float &z) const { const float2 v = a[i]; y = v.x; z = v.y; }
    __device__ __forceinline__ void eg(int i, float &e, float &gy, float &gz) const
    {
        const float4 v = f[i];
        e = v.x; gy = v.y; gz = v.z;
    }
    __device__ __forceinline__ void store(int i, double ay, double az, double e, double gy, double gz)
    {
        a[i] = make_float2((float)ay, (float)az);
        f[i] = make_float4((float)e, (float)gy, (float)gz, 0.f);
    }
    __device__ __forceinline__ void copy_image(int i, const StageImages &img, int g)
    {
        a[i] = img.a[g];
        f[i] = img.f[g];
    }
    static size_t bytes(size_t W) { return W * (sizeof(float2) + sizeof(float4)); }
};
// Double form: the differences a_j - a_{j-1} are formed from the staged
// coefficients when read (the same double values a staged copy would hold), which
// keeps the tile within shared memory for M = 4096, k = 5.
template <> struct FieldTile<double> {
    double2 *a;     // (a_y, a_z)
    double *e;      // ebar dx
    __device__ __forceinline__ void aa(int i, double &y, double &z) const { const double2 v = a[i]; y = v.x; z = v.y; }
    __device__ __forceinline__ void eg(int i, double &ev, double &gy, double &gz) const
    {
        const double2 v = a[i], w = a[i - 1];
        ev = e[i]; gy = v.x - w.x; gz = v.y - w.y;
    }
    __device__ __forceinline__ void store(int i, double ay, double az, double ev, double, double)
    {
        a[i] = make_double2(ay, az);
        e[i] = ev;
    }
    __device__ __forceinline__ void copy_image(int, const StageImages &, int) {}
    static size_t bytes(size_t W) { return W * (sizeof(double2) + sizeof(double)); }
};

template <typename R>
__device__ __forceinline__ FieldTile<R> carve_tile(unsigned char *p, int W);
template <>
__device__ __forceinline__ FieldTile<float> carve_tile<float>(unsigned char *p, int W)
{
    FieldTile<float> t;
    t.f = reinterpret_cast<float4 *>(p);
    t.a = reinterpret_cast<float2 *>(t.f + W);
    return t;
}
template <>
__device__ __forceinline__ FieldTile<double> carve_tile<double>(unsigned char *p, int W)
{
    FieldTile<double> t;
    t.a = reinterpret_cast<double2 *>(p);
    t.e = reinterpret_cast<double *>(t.a + W);
    return t;
}

// Correctly rounded division: an approximate reciprocal carries a systematic
// bias that the discrete-gradient identity turns into a steady energy drift.
template <typename R> __device__ __forceinline__ R fdiv_(R a, R b) { return a / b; }

// Contiguous chunk of markers owned by one block (a multiple of 32, so every
// warp's lanes see consecutive, sorted markers).
__device__ __forceinline__ void block_chunk(long long np, long long &beg, long long &end)
{
    long long chunk = (np + gridDim.x - 1) / gridDim.x;
    chunk = (chunk + 31) & ~31LL;
    beg = (long long)blockIdx.x * chunk;
    end = beg + chunk < np ? beg + chunk : np;
}

// Markers stream through shared memory in tiles of kTile, NS tiles in flight.
// The block's q-th tile overall goes to stage q % NS.  Each stage has a
// "full" mbarrier (completed by the bulk copies of its arrays, cp.async.bulk)
// and an "empty" mbarrier (one arrival per warp once the warp has read it).
// Warps do not synchronise with each other per tile: a warp waits only for its
// next tile to land, and thread 0 refills a stage once every warp has released
// it.  A block may process several ranges (batched runs); q runs on across
// them, so the barrier phases stay consistent.  Every wait is bounded; a wait
// that gives up sets the block's abort flag, after which no warp consumes or
// issues more tiles, and the copies still in flight are waited for (bounded)
// before the block leaves.  The marker arrays are allocated with padding, so a
// tile's byte count may be rounded up to a multiple of 16.
constexpr int kTileU = 1;                      // markers per thread per tile
constexpr int kTile = kSweepThreads * kTileU;  // markers per tile
constexpr int kMaxStages = 4;
constexpr int kSweepWarps = kSweepThreads / 32;
// stages in flight: 4 in float, 2 in double (whose tiles are twice as large and
// whose field staging needs the room at M = 4096)
template <typename R> struct Stages { static constexpr int n = Real<R>::fp32 ? 4 : 2; };
inline int stage_count(int fp32) { return fp32 ? 4 : 2; }

struct TileBars {
    unsigned long long full[kMaxStages];
    unsigned long long empty[kMaxStages];
    int abort;
    unsigned long long issued;      // tiles issued by this block so far (thread 0)
};
static_assert(sizeof(TileBars) <= 128, "tile barriers live in the first 128 bytes");

__device__ __forceinline__ void tile_bars_init(TileBars &B)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(&B.full[s], 1);
            mbar_init(&B.empty[s], kSweepWarps);
        }
        B.abort = 0;
        B.issued = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

__device__ __forceinline__ bool tile_aborted(const TileBars &B)
{
    return __shfl_sync(0xffffffffu, *reinterpret_cast<const volatile int *>(&B.abort), 0) != 0;
}

// Warp: wait (bounded) for tile q; false (warp-uniform) after a timeout or an abort.
template <int NS>
__device__ __forceinline__ bool tile_acquire(TileBars &B, unsigned long long q)
{
    if (tile_aborted(B)) return false;
    const bool ok = mbar_wait(&B.full[q % NS], (unsigned)((q / NS) & 1));
    if (__all_sync(0xffffffffu, ok)) return true;
    if ((threadIdx.x & 31) == 0) atomicExch(&B.abort, 1);
    return false;
}

// Warp: done reading tile q.
template <int NS>
__device__ __forceinline__ void tile_release(TileBars &B, unsigned long long q)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&B.empty[q % NS]);
}

// Thread 0: may tile q be written into its stage?  Waits (bounded) until every
// warp released the stage's previous tile q - NS.
template <int NS>
__device__ __forceinline__ bool tile_stage_free(TileBars &B, unsigned long long q)
{
    if (q < (unsigned long long)NS) return true;
    if (mbar_wait(&B.empty[q % NS], (unsigned)(((q / NS) - 1) & 1))) return true;
    atomicExch(&B.abort, 1);
    return false;
}

// Thread 0, after the block's warps left the range: wait (bounded) for the bulk
// copies of the last tiles issued, so none is in flight when shared memory is reused
// or the block exits.
template <int NS>
__device__ __forceinline__ void tile_drain(TileBars &B)
{
    const unsigned long long n = B.issued;
    for (unsigned long long q = n > (unsigned long long)NS ? n - NS : 0; q < n; ++q)
        mbar_wait(&B.full[q % NS], (unsigned)((q / NS) & 1));
}

// ---------------------------------------------------------------------------
// Subsystem I: one Picard sweep (Sec. 4.2).  Per marker, with x^n = (c0, t0),
// the iterate x^(k) = x^n + delta^(k) and ebar = (e^n + e^(k))/2:
//   A0 = A_h(x^n), A1 = A_h(x^(k)), m = path means of Lambda^1 on x^n -> x^(k),
//   Ebar = sum m ebar, D = sum m (G a)  [= (A1-A0)/(x^(k)-x^n), exact],
//   p^(k+1) = p^n + dt Ebar - dt (A1+A0).D / (g(p^n,A1) + g(p^n,A0)),
//   delta^(k+1) = dt (p^n + p^(k+1)) / (g(p^n,A1) + g(p^(k+1),A1)) / dx,
//   j_i += w int_{x^n}^{x^n+delta^(k+1)} Lambda^1_i.
// In cell units with tau = dt/dx: p^(k+1) = p^n + tau (Ebar dx - (A1+A0).D dx/(...)).
// ---------------------------------------------------------------------------
// Markers [beg, end) of one run.  q = the block's tile sequence number (in/out).
// Returns false after a bounded wait gave up (the block must then stop).
// Start-point cache of subsystem I: (A_y, A_z, gamma, unused) per marker, as one
// 16-byte (float) or two 16-byte (double) accesses.
template <typename R>
__device__ __forceinline__ void start_cache_store(void *base, long long a, R y, R z, R g)
{
    if constexpr (Real<R>::fp32) {
        reinterpret_cast<float4 *>(base)[a] = make_float4(y, z, g, 0.f);
    } else {
        double2 *q = reinterpret_cast<double2 *>(base) + 2 * a;
        q[0] = make_double2(y, z);
        q[1] = make_double2(g, 0.0);
    }
}

template <typename R>
__device__ __forceinline__ void start_cache_load(const void *base, long long a, R &y, R &z, R &g)
{
    if constexpr (Real<R>::fp32) {
        const float4 v = reinterpret_cast<const float4 *>(base)[a];
        y = v.x;
        z = v.y;
        g = v.z;
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(base) + 2 * a;
        const double2 u = q[0], w = q[1];
        y = u.x;
        z = u.y;
        g = w.x;
    }
}

// Deposit of one marker's path integral as a difference of the cumulative sums
// C_i(x) = sum_{j >= i} Lambda^0_j(x) at its two ends (see sweep1_range):
// S0, S1 are the partial sums at x^n (cell c0) and x^(k+1) (cell c0 + n), in
// the scaled units of bspline_scaled.  For |n| <= kCdMax the nonzero values lie
// on the KB = K + kCdMax nodes a - r (a = max(c0, c0 + n)) and go into the warp
// window as one block:  val[r] = C(S1, r - nl) - C(S0, r - nr), nl = max(0, -n),
// nr = max(0, n), C(S, i) = 0 (i < 0), S[i] (i < K), K! (i >= K).  Longer paths
// (rare) add the same values node by node to the shared row.
constexpr int kCdMax = 2;

template <int K, int NL, int NR, typename R>
__device__ __forceinline__ void cdiff_block(const R *S0, const R *S1, R *val)
{
    constexpr int KB = K + kCdMax;
    const R one = R(Fact<K>::v);
#pragma unroll
    for (int r = 0; r < KB; ++r) {
        const int i1 = r - NL, i0 = r - NR;
        const R c1 = i1 < 0 ? R(0) : (i1 < K ? S1[i1 < K ? i1 : 0] : one);
        const R c0 = i0 < 0 ? R(0) : (i0 < K ? S0[i0 < K ? i0 : 0] : one);
        val[r] = c1 - c0;
    }
}

template <int K, class Win, typename R>
__device__ __forceinline__ void deposit_cdiff(Win &win, const R *S0, const R *S1, int n, int c0, int wb, int H,
                                              double *s_acc, double wdx)
{
    constexpr int KB = K + kCdMax;
    R val[KB];
    switch (n) {
    case -2: cdiff_block<K, 2, 0>(S0, S1, val); break;
    case -1: cdiff_block<K, 1, 0>(S0, S1, val); break;
    case 0: cdiff_block<K, 0, 0>(S0, S1, val); break;
    case 1: cdiff_block<K, 0, 1>(S0, S1, val); break;
    case 2: cdiff_block<K, 0, 2>(S0, S1, val); break;
    default: {
        // a path across more than kCdMax knots: node by node into the shared row
        const int nl = n < 0 ? -n : 0, nr = n > 0 ? n : 0;
        const int a = c0 + nr;
        const R one = R(Fact<K>::v);
        for (int r = 0; r < K + nl + nr; ++r) {
            const int i1 = r - nl, i0 = r - nr;
            R c1 = R(0), cc0 = R(0);
#pragma unroll
            for (int q = 0; q < K; ++q) {
                if (i1 == q) c1 = S1[q];
                if (i0 == q) cc0 = S0[q];
            }
            if (i1 >= K) c1 = one;
            if (i0 >= K) cc0 = one;
            const R d = c1 - cc0;
            if (d != R(0)) atomicAdd(&s_acc[a - r + H], wdx * (double)d);
        }
        return;
    }
    }
    const int a = c0 + (n > 0 ? n : 0);
    if (!win.put(a - wb, val)) {
#pragma unroll
        for (int r = 0; r < KB; ++r)
            if (val[r] != R(0)) atomicAdd(&s_acc[a - r + H], wdx * (double)val[r]);
    }
}

// PRE: the predicted start instead of a sweep -- the proposal delta^(0) (the
// explicit predictor when A.warm, else the one already in delta) is written back
// and its path current deposited into A.j; no gather walk, no momentum update.
template <int K, typename R, int ACC, bool PRE = false>
__device__ __forceinline__ bool sweep1_range(const Sweep1Args &A, long long beg, long long end,
                                             unsigned char *smem, unsigned long long &q)
{
    constexpr int NS = Stages<R>::n;
    const int H = A.H;
    const int W = A.M + 2 * H;
    TileBars &Bars = *reinterpret_cast<TileBars *>(smem);
    unsigned char *st = smem + 128;
    // stage b: cell[kTile], t[kTile], p[kTile], delta[kTile]
    unsigned char *const stage0 = st;
    constexpr size_t kStageBytes = kTile * (sizeof(int32_t) + 3 * sizeof(R));
    auto s_cell = [&](int b) { return reinterpret_cast<int32_t *>(stage0 + b * kStageBytes); };
    auto s_t = [&](int b) { return reinterpret_cast<R *>(stage0 + b * kStageBytes + kTile * sizeof(int32_t)); };
    auto s_p = [&](int b) { return s_t(b) + kTile; };
    auto s_d = [&](int b) { return s_t(b) + 2 * kTile; };
    st += NS * kStageBytes;
    double *s_acc = reinterpret_cast<double *>(st);
    double *s_red = s_acc + W;
    FieldTile<R> F = carve_tile<R>(reinterpret_cast<unsigned char *>(s_red + 32), W);

    const long long ntile = end > beg ? (end - beg + kTile - 1) / kTile : 0;
    const unsigned long long q0 = q, qend = q + (unsigned long long)ntile;
    double *jout = A.j;
    bool warm = A.warm != 0;
    bool first = A.first != 0;
    if (!PRE && A.graph) {                  // replayed by a graph: buffers by sweep parity
        const int it = *reinterpret_cast<volatile const int *>(&A.ctrl->iter);
        jout = A.jpair[it & 1];
        warm = warm && it == 0;
        first = it == 0;
    }
    const bool need_delta = !warm;
    auto issue = [&](long long i) {            // thread 0: copies of tile i into stage (q0 + i) % NS
        if (*reinterpret_cast<volatile int *>(&Bars.abort) || !tile_stage_free<NS>(Bars, q0 + i)) return;
        const long long s0 = beg + i * kTile;
        long long n = end - s0 < kTile ? end - s0 : kTile;
        n = (n + 3) & ~3LL;
        const int b = (int)((q0 + i) % NS);
        const unsigned bi = (unsigned)(n * sizeof(int32_t)), br = (unsigned)(n * sizeof(R));
        fence_proxy_async();
        mbar_expect_tx(&Bars.full[b], bi + 2 * br + (need_delta ? br : 0u));
        bulk_g2s(s_cell(b), A.P.cell + s0, bi, &Bars.full[b]);
        bulk_g2s(s_t(b), static_cast<const R *>(A.P.t) + s0, br, &Bars.full[b]);
        bulk_g2s(s_p(b), static_cast<const R *>(A.P.p) + s0, br, &Bars.full[b]);
        if (need_delta) bulk_g2s(s_d(b), static_cast<const R *>(A.P.delta) + s0, br, &Bars.full[b]);
        Bars.issued = q0 + i + 1;
    };
    __syncthreads();                           // shared memory of a previous range is free
    if (threadIdx.x == 0)
        for (long long i = 0; i < ntile && i < NS; ++i) issue(i);

    // scaled arithmetic (see piece_means_scaled): the basis is K! N^K, the path
    // means are S1 = S_{K-1} times the means of N^{K-1}; so the staged fields are
    // a / K! and ebar dx / S1, the A-term sum is multiplied by K!/S1 = DK, and the
    // deposit by w dx / S1 when flushed
    constexpr int S1 = MeanScale<K - 1>::S;
    constexpr int DK = K / MeanScale<K - 1>::X;
    const double inv_fact = 1.0 / (double)Fact<K>::v;
    if (Real<R>::fp32 && A.img.a) {
        // float images built on the grid side (same values as the branch below)
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            const int g = wrap_cell(i - H, A.M);
            F.copy_image(i, A.img, g);
            s_acc[i] = 0.0;
        }
    } else {
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            const int g = wrap_cell(i - H, A.M);
            const int gm = g == 0 ? A.M - 1 : g - 1;
            // the differences of a are formed from the coefficients as staged (rounded
            // to R), so that the path mean of dA/dx times (x1 - x0) equals A(x1) - A(x0)
            // of the staged field: the discrete gradient of the A-term stays exact for
            // the field the markers see
            const R ay = (R)(A.ay[g] * inv_fact), aym = (R)(A.ay[gm] * inv_fact);
            const R az = (R)(A.az[g] * inv_fact), azm = (R)(A.az[gm] * inv_fact);
            F.store(i, ay, az, A.ebar[g] * A.dx / S1, (double)(ay - aym), (double)(az - azm));
            s_acc[i] = 0.0;
        }
    }
    __syncthreads();

    R *__restrict__ dp = static_cast<R *>(A.P.delta);
    R *__restrict__ pnp = static_cast<R *>(A.P.pnew);
    const R tau = (R)(A.dt / A.dx);
    const double wdx = A.w * A.dx * inv_fact;   // deposit flush scale (C in units of K!)
    const R dlim = (R)A.Dlim;
    const R one = R(1);
    R dmax = R(0);
    bool bad = false;
    // window: blocks of KB = K + kCdMax values anchored at the larger end cell,
    // max(c0, c1) - wb in [0, 3]; V1 nodes wb - KB + 1 .. wb + 3
    constexpr int KB = K + kCdMax;
    DepWindow<R, KB + 3, KB, KB - 1, 0, 3, typename AccOf<R, ACC, K>::T> win;
    win.clear();
    int wb = INT_MIN;

    for (long long i = 0; i < ntile; ++i) {
        if (!tile_acquire<NS>(Bars, q0 + i)) break;
        const int b = (int)((q0 + i) % NS);
        const long long s0 = beg + i * kTile;
#pragma unroll 1
        for (int u = 0; u < kTileU; ++u) {
            const int jl = u * kSweepThreads + threadIdx.x;
            const long long a = s0 + jl;
            const bool act = a < end;
            // reach above the cell: the path (Dlim cells)
            const int c0 = warp_unwrap_cell(act ? s_cell(b)[jl] : 0, act, A.M, H - A.Dlim);
            const int lead = __reduce_min_sync(0xffffffffu, act ? c0 : INT_MAX);
            if (lead == INT_MAX) break;                    // whole warp past the chunk end
            if (lead != wb) {
                if (wb != INT_MIN) win.advance(lead - wb, s_acc, wb - (KB - 1) + H, wdx);
                wb = lead;
            }
            const unsigned amask = __ballot_sync(0xffffffffu, act);
            if (!act) continue;
            const R t0 = s_t(b)[jl];
            const R pn = s_p(b)[jl];
            // basis at the start point: A(x^n) and the partial sums of the deposit
            R v0[K + 1];
            bspline_scaled<K, R>(t0, v0);
            // A(x^n) and gamma(p^n, A(x^n)) do not change during the loop: in the
            // double form the first sweep stores them and the later ones read them
            // back (the float form recomputes: there the extra bytes cost more)
            R A0y = R(0), A0z = R(0), g0;
            bool cached = false;
            if constexpr (!Real<R>::fp32 && !PRE) cached = !first && A.a0 != nullptr;
            if (cached) {
                start_cache_load<R>(A.a0, a, A0y, A0z, g0);
            } else {
#pragma unroll
                for (int r = 0; r <= K; ++r) {
                    R y, z;
                    F.aa(c0 - r + H, y, z);
                    A0y += y * v0[r];
                    A0z += z * v0[r];
                }
                g0 = sqrt_(one + pn * pn + A0y * A0y + A0z * A0z);
                if constexpr (!Real<R>::fp32 && !PRE)
                    if (A.a0) start_cache_store<R>(A.a0, a, A0y, A0z, g0);
            }
            R dold = warm ? fdiv_(tau * pn, g0) : s_d(b)[jl];
            if (!(fabs(dold) <= dlim)) { bad = true; dold = R(0); }
            R dnew = R(0), pnew = R(0);
            if constexpr (PRE) {
                dnew = dold;
            } else {
                // Path integrals along x^n -> x^(k) (cell units), unnormalised:
                //   EI = int ebar dt,  DI = int dA/dt dt / DK,
                // the path means being EI/dold and DK DI/dold (the means at t0 when
                // dold = 0).  A(x^(k)) = A(x^n) + DK DI exactly for the staged field (the
                // staged differences of a are those of the staged coefficients), so the
                // end point needs no basis evaluation of its own.
                R EI = R(0), DIy = R(0), DIz = R(0);
                const bool still = dold == R(0);
                const int n1 = __reduce_max_sync(amask, path_pieces(t0, dold));
                walk_uniform<K, R>(t0, dold, n1, [&](int c, R h, const R *m, int p) {
                    R e = R(0), gy = R(0), gz = R(0);
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        R ev, y, z;
                        F.eg(c0 + c - r + H, ev, y, z);
                        e += m[r] * ev;
                        gy += m[r] * y;
                        gz += m[r] * z;
                    }
                    const R hw = still ? (p == 0 ? one : R(0)) : h;
                    EI += hw * e;
                    DIy += hw * gy;
                    DIz += hw * gz;
                });
                const R dn = still ? one : dold;
                const R A1y = A0y + R(DK) * (still ? R(0) : DIy);
                const R A1z = A0z + R(DK) * (still ? R(0) : DIz);

                // p^(k+1) = p^n + tau (Ebar - (A1 + A0).D / (g1 + g0)) with Ebar = EI/dn,
                // D = DK DI/dn, as one division
                const R q1 = one + A1y * A1y + A1z * A1z;
                const R g1 = sqrt_(q1 + pn * pn);
                const R G = g1 + g0;
                const R num = EI * G - R(DK) * ((A1y + A0y) * DIy + (A1z + A0z) * DIz);
                R spin_term = R(0);
                if constexpr (!Real<R>::fp32) {
                    if (A.hbar != 0.0) {
                        // discrete gradient of the Zeeman energy: D2 = path mean of d^2A/dx^2
                        // along x^n -> x^(k) (the exact difference quotient of dA/dx; its
                        // limit at rest is the point value), from the second differences of
                        // the staged coefficients and the means of the degree-(K-2) pieces
                        const int id = A.P.id[a];
                        double D2y = 0.0, D2z = 0.0;
                        const double invd = still ? 0.0 : 1.0 / dold;
                        walk_path<K - 1, double>(t0, dold, [&](int c, double h, const double *m2, bool single) {
                            double gy = 0.0, gz = 0.0;
#pragma unroll
                            for (int r = 0; r <= K - 2; ++r) {
                                const int i = c0 + c - r + H;
                                double y0, z0, y1, z1, y2, z2;
                                F.aa(i, y0, z0);
                                F.aa(i - 1, y1, z1);
                                F.aa(i - 2, y2, z2);
                                gy += m2[r] * ((y0 - y1) - (y1 - y2));
                                gz += m2[r] * ((z0 - z1) - (z1 - z2));
                            }
                            const double f = single ? 1.0 : h * invd;
                            D2y += f * gy;
                            D2z += f * gz;
                        });
                        // staged coefficients are a / K!; D2 is per cell^2, the update per dx
                        const double fac = (double)Fact<K>::v / A.dx;
                        spin_term = A.hbar * fac * (A.sy[id] * D2z - A.sz[id] * D2y);
                    }
                }
                pnew = pn + tau * (fdiv_(num, dn * G) - spin_term);
                const R g2 = sqrt_(q1 + pnew * pnew);
                dnew = fdiv_(tau * (pn + pnew), g1 + g2);
                if (!(fabs(dnew) <= dlim)) { bad = true; dnew = R(0); }
            }

            // Deposit j_i += w int_{x^n}^{x^(k+1)} Lambda^1_i = w dx (C_i(x^(k+1)) - C_i(x^n))
            // with C_i(x) = sum_{j >= i} Lambda^0_j(x): the derivative relation of Sec. 3.1
            // telescoped (the identity behind the paper's discrete Gauss law).  In a
            // cell c at offset t, C_{c-r} = S[r] = sum_{r' <= r} N^K(r' + t) for
            // r < K, 1 below, 0 above; here in the scaled units of bspline_scaled
            // (K! N^K, so "1" is K!).  The end point's cell is that of finalize.
            {
                const R s1 = t0 + dnew;
                const R f1 = floor_(s1);
                int n = (int)f1;
                R t1 = s1 - f1;
                if (t1 >= one) { t1 = R(0); n += 1; }
                R v1[K + 1];
                bspline_scaled<K, R>(t1, v1);
                R S0[K], S1[K];
                S0[0] = v0[0];
                S1[0] = v1[0];
#pragma unroll
                for (int r = 1; r < K; ++r) {
                    S0[r] = S0[r - 1] + v0[r];
                    S1[r] = S1[r - 1] + v1[r];
                }
                deposit_cdiff<K>(win, S0, S1, n, c0, wb, H, s_acc, wdx);
            }
            if constexpr (PRE) {
                dp[a] = dnew;
            } else {
                R inc = fabs(dnew - dold);
                if (Real<R>::fp32) inc = __fdividef(inc, fmax(one, fabs(dnew)));   // convergence metric only
                dmax = (inc > dmax || inc != inc) ? inc : dmax;
                dp[a] = dnew;
                pnp[a] = pnew;
            }
        }
        tile_release<NS>(Bars, q0 + i);
        if (threadIdx.x == 0 && i + NS < ntile) issue(i + NS);
    }
    if (wb != INT_MIN) win.flush(s_acc, wb - (KB - 1) + H, wdx);
    if (bad) atomicOr(&A.ctrl->status, STATUS_NUMERIC);
    __syncthreads();
    const bool timeout = *reinterpret_cast<volatile int *>(&Bars.abort) != 0;
    if (timeout && threadIdx.x == 0) {
        atomicOr(&A.ctrl->status, STATUS_TIMEOUT);
        tile_drain<NS>(Bars);
    }
    if (!PRE) block_max_to(&A.ctrl->dmax_bits, (double)dmax, s_red);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const double val = s_acc[i];
        if (val != 0.0) atomicAdd(&jout[wrap_cell(i - H, A.M)], val);
    }
    q = qend;
    return !timeout;
}

template <int K, typename R, int ACC>
__global__ void __launch_bounds__(kSweepThreads, Real<R>::fp32 ? 2 : 1) k_sweep1(Sweep1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    tile_bars_init(*reinterpret_cast<TileBars *>(smem));
    long long beg, end;
    block_chunk(A.np, beg, end);
    unsigned long long q = 0;
    sweep1_range<K, R, ACC>(A, beg, end, smem, q);
}

// ---------------------------------------------------------------------------
// Start of subsystem I with a predicted field: the proposal x^(0) = x^n + delta^(0)
// (the explicit predictor dt p^n / gamma(p^n, A(x^n)), written here, or the learned
// one already in delta) and its path-integrated current j^(0), deposited as in the
// sweeps, so that the fixed-point loop can start from e^(0) = e^n - M1^{-1} j^(0),
// the field consistent with x^(0).  The fixed point does not depend on the start;
// the starting field sets how far the first sweep's kick is off.
// ---------------------------------------------------------------------------
template <int K, typename R, int ACC>
__global__ void __launch_bounds__(kSweepThreads, Real<R>::fp32 ? 2 : 1) k_predeposit(Sweep1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    tile_bars_init(*reinterpret_cast<TileBars *>(smem));
    long long beg, end;
    block_chunk(A.np, beg, end);
    unsigned long long q = 0;
    sweep1_range<K, R, ACC, true>(A, beg, end, smem, q);
}

size_t sweep1_smem(int M, int H, int fp32)
{
    const size_t W = (size_t)M + 2 * (size_t)H;
    const size_t stages = (size_t)stage_count(fp32) * kTile * (sizeof(int32_t) + 3 * (fp32 ? sizeof(float) : sizeof(double)));
    return 128 + stages + (W + 32) * sizeof(double) +
           (fp32 ? FieldTile<float>::bytes(W) : FieldTile<double>::bytes(W));
}

// Instantiations: double form with double windows; float form with compensated
// windows for every degree, and with plain float or double windows (kept to
// compare the deposit accumulations) for k = 3 and 5.
#define PIC_FOR_SWEEP_VARIANTS(X)                                                                   \
    X(2, double, ACC_NATIVE) X(3, double, ACC_NATIVE) X(4, double, ACC_NATIVE) X(5, double, ACC_NATIVE) \
    X(2, float, ACC_COMP) X(3, float, ACC_COMP) X(4, float, ACC_COMP) X(5, float, ACC_COMP)             \
    X(3, float, ACC_NATIVE) X(5, float, ACC_NATIVE) X(3, float, ACC_DOUBLE) X(5, float, ACC_DOUBLE)

bool sweep_variant_ok(int K, int fp32, int acc)
{
#define OKV(KK, RR, AA) if (K == KK && (fp32 != 0) == std::is_same<RR, float>::value && acc == AA) return true;
    PIC_FOR_SWEEP_VARIANTS(OKV)
#undef OKV
    return false;
}

int launch_sweep1(const Sweep1Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
#define L1(KK, RR, AA)                                                                              \
    if (a.K == KK && (a.fp32 != 0) == std::is_same<RR, float>::value && a.acc == AA) {              \
        k_sweep1<KK, RR, AA><<<grid, block, smem, s>>>(a);                                          \
        return 0;                                                                                   \
    }
    PIC_FOR_SWEEP_VARIANTS(L1)
#undef L1
    return 1;
}

// ---------------------------------------------------------------------------
// Path-integrated current of given displacements (pic_deposit CURRENT): the
// deposit half of the sweep above, in the form's precision.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256) k_current(CurrentArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int H = A.H;
    const int W = A.M + 2 * H;
    double *s_acc = reinterpret_cast<double *>(smem);
    for (int i = threadIdx.x; i < W; i += blockDim.x) s_acc[i] = 0.0;
    __syncthreads();
    const R *tp = static_cast<const R *>(A.P.t);
    const double wdx = A.w * A.dx / MeanScale<K - 1>::S;   // walk_uniform returns scaled means
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c0 = A.P.cell[a];
        const R t0 = tp[a];
        R d = (R)(A.disp[A.P.id[a]] / A.dx);
        if (!(fabs(d) <= (R)A.Dlim)) { bad = true; continue; }
        walk_uniform<K, R>(t0, d, path_pieces(t0, d), [&](int c, R h, const R *m, int) {
#pragma unroll
            for (int r = 0; r < K; ++r) atomicAdd(&s_acc[c0 + c - r + H], wdx * (double)(h * m[r]));
        });
    }
    if (bad) atomicOr(&A.ctrl->status, STATUS_NUMERIC);
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const double v = s_acc[i];
        if (v != 0.0) atomicAdd(&A.out[wrap_cell(i - H, A.M)], v);
    }
}

template <typename R>
static int launch_current_t(const CurrentArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    switch (a.K) {
    case 2: k_current<2, R><<<grid, block, smem, s>>>(a); break;
    case 3: k_current<3, R><<<grid, block, smem, s>>>(a); break;
    case 4: k_current<4, R><<<grid, block, smem, s>>>(a); break;
    case 5: k_current<5, R><<<grid, block, smem, s>>>(a); break;
    default: return 1;
    }
    return 0;
}

int launch_current(const CurrentArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    return a.fp32 ? launch_current_t<float>(a, grid, block, smem, s)
                  : launch_current_t<double>(a, grid, block, smem, s);
}

// ---------------------------------------------------------------------------
// Subsystem II: one fixed-point sweep (Sec. 4.2).  Markers frozen at x; with
// A0 = A^n_h(x), A1 = A^(k)_h(x):
//   s_i += w (A0 + A1) Lambda^0_i(x) / (g(p,A0) + g(p,A1))   (y and z);
// the weight w enters at the window flush, in double.  Same tile pipeline
// (bulk copies of cell, t, p two tiles ahead) as the subsystem-I sweep.
// ---------------------------------------------------------------------------
template <int K, typename R, int ACC>
__device__ __forceinline__ bool sweep2_range(const Sweep2Args &A, long long beg, long long end,
                                             unsigned char *smem, unsigned long long &q)
{
    constexpr int NS = Stages<R>::n;
    const int H = A.H;
    const int W = A.M + 2 * H;
    TileBars &Bars = *reinterpret_cast<TileBars *>(smem);
    unsigned char *st = smem + 128;
    // stage b: cell[kTile], t[kTile], p[kTile]
    unsigned char *const stage0 = st;
    constexpr size_t kStageBytes = kTile * (sizeof(int32_t) + 2 * sizeof(R));
    auto s_cell = [&](int b) { return reinterpret_cast<int32_t *>(stage0 + b * kStageBytes); };
    auto s_t = [&](int b) { return reinterpret_cast<R *>(stage0 + b * kStageBytes + kTile * sizeof(int32_t)); };
    auto s_p = [&](int b) { return s_t(b) + kTile; };
    st += NS * kStageBytes;
    double *s_sy = reinterpret_cast<double *>(st);
    double *s_sz = s_sy + W;
    using R2 = typename std::conditional<std::is_same<R, float>::value, float2, double2>::type;
    R2 *s_an = reinterpret_cast<R2 *>(s_sz + W);
    R2 *s_ak = s_an + W;
    // float form: the rounding residues of a^n + a^(k) per node (see below)
    float2 *s_lo = reinterpret_cast<float2 *>(s_ak + W);

    const long long ntile = end > beg ? (end - beg + kTile - 1) / kTile : 0;
    const unsigned long long q0 = q, qend = q + (unsigned long long)ntile;
    auto issue = [&](long long i) {            // thread 0: copies of tile i into stage (q0 + i) % NS
        if (*reinterpret_cast<volatile int *>(&Bars.abort) || !tile_stage_free<NS>(Bars, q0 + i)) return;
        const long long s0 = beg + i * kTile;
        long long n = end - s0 < kTile ? end - s0 : kTile;
        n = (n + 3) & ~3LL;
        const int b = (int)((q0 + i) % NS);
        const unsigned bi = (unsigned)(n * sizeof(int32_t)), br = (unsigned)(n * sizeof(R));
        fence_proxy_async();
        mbar_expect_tx(&Bars.full[b], bi + 2 * br);
        bulk_g2s(s_cell(b), A.P.cell + s0, bi, &Bars.full[b]);
        bulk_g2s(s_t(b), static_cast<const R *>(A.P.t) + s0, br, &Bars.full[b]);
        bulk_g2s(s_p(b), static_cast<const R *>(A.P.p) + s0, br, &Bars.full[b]);
        Bars.issued = q0 + i + 1;
    };
    __syncthreads();                           // shared memory of a previous range is free
    if (threadIdx.x == 0)
        for (long long i = 0; i < ntile && i < NS; ++i) issue(i);
    // scaled basis K! N^K: coefficients staged as a / K!, deposits flushed times w / K!
    const double inv_fact = 1.0 / (double)Fact<K>::v;
    if constexpr (Real<R>::fp32) {
        if (A.img.an) {
            // float images built on the grid side (same values as the branch below)
            for (int i = threadIdx.x; i < W; i += blockDim.x) {
                const int g = wrap_cell(i - H, A.M);
                s_an[i] = A.img.an[g];
                s_ak[i] = A.img.ak[g];
                s_lo[i] = A.img.lo[g];
                s_sy[i] = 0.0;
                s_sz[i] = 0.0;
            }
        }
    }
    for (int i = threadIdx.x; i < W && !(Real<R>::fp32 && A.img.an); i += blockDim.x) {
        const int g = wrap_cell(i - H, A.M);
        const double ny = A.an_y[g] * inv_fact, nz = A.an_z[g] * inv_fact;
        const double ky = A.ak_y[g] * inv_fact, kz = A.ak_z[g] * inv_fact;
        s_an[i].x = (R)ny;
        s_an[i].y = (R)nz;
        s_ak[i].x = (R)ky;
        s_ak[i].y = (R)kz;
        if constexpr (Real<R>::fp32) {
            // The float rounding of a coefficient is the same for every marker near
            // its node, so it does not average out over markers: in the exchange
            // term (A1 - A0)(A1 + A0)/(g0 + g1) it shows as an energy error of
            // about 1e-11 per step.  The residues of the sum a^n + a^(k) are kept
            // and enter the numerator before its one rounding, which leaves only
            // per-marker rounding (unbiased on average).
            s_lo[i] = make_float2((float)((ny - (double)s_an[i].x) + (ky - (double)s_ak[i].x)),
                                  (float)((nz - (double)s_an[i].y) + (kz - (double)s_ak[i].y)));
        }
        s_sy[i] = 0.0;
        s_sz[i] = 0.0;
    }
    __syncthreads();
    const double w = A.w * inv_fact;
    const R one = R(1);
    // window: marker cells wb .. wb+2 (wb = the warp's lowest), V0 nodes wb-K .. wb+2
    DepWindow<R, K + 3, K + 1, K, 0, 2, typename AccOf<R, ACC, K>::T> wy;
    DepWindow<R, K + 3, K + 1, K, 0, 2, typename AccOf<R, ACC, K>::T, true> wz;
    wy.clear();
    wz.clear();
    int wb = INT_MIN;
    for (long long i = 0; i < ntile; ++i) {
        if (!tile_acquire<NS>(Bars, q0 + i)) break;
        const int b = (int)((q0 + i) % NS);
        const long long s0 = beg + i * kTile;
#pragma unroll 1
        for (int u = 0; u < kTileU; ++u) {
            const int jl = u * kSweepThreads + threadIdx.x;
            const long long a = s0 + jl;
            const bool act = a < end;
            const int c = warp_unwrap_cell(act ? s_cell(b)[jl] : 0, act, A.M, H);   // no reach above
            const int lead = __reduce_min_sync(0xffffffffu, act ? c : INT_MAX);
            if (lead == INT_MAX) break;
            if (lead != wb) {
                if (wb != INT_MIN) {
                    wy.advance(lead - wb, s_sy, wb - K + H, w);
                    wz.advance(lead - wb, s_sz, wb - K + H, w);
                }
                wb = lead;
            }
            if (!act) continue;
            const R t = s_t(b)[jl];
            const R p = s_p(b)[jl];
            R v[K + 1];
            bspline_scaled<K, R>(t, v);
            R A0y = R(0), A0z = R(0), A1y = R(0), A1z = R(0);
#pragma unroll
            for (int r = 0; r <= K; ++r) {
                const R2 an = s_an[c - r + H], ak = s_ak[c - r + H];
                A0y += an.x * v[r];
                A0z += an.y * v[r];
                A1y += ak.x * v[r];
                A1z += ak.y * v[r];
            }
            const R pp1 = one + p * p;
            const R g0 = sqrt_(pp1 + A0y * A0y + A0z * A0z);
            const R g1 = sqrt_(pp1 + A1y * A1y + A1z * A1z);
            R Ly = R(0), Lz = R(0);
            if constexpr (Real<R>::fp32) {
#pragma unroll
                for (int r = 0; r <= K; ++r) {
                    const float2 l = s_lo[c - r + H];
                    Ly += l.x * v[r];
                    Lz += l.y * v[r];
                }
            }
            const R cf = fdiv_(one, g0 + g1);
            const R sy = A0y + A1y, sz = A0z + A1z;
            R fy, fz;
            if constexpr (Real<R>::fp32) {
                // f = cf (s + L) rounded once: the residue L is far below half an ulp
                // of s, so s + L in float would drop it.  The product's own rounding
                // error (exact by an fma) and cf L are added before the one rounding.
                const float py = cf * sy, pz = cf * sz;
                fy = py + (fmaf(cf, sy, -py) + cf * Ly);
                fz = pz + (fmaf(cf, sz, -pz) + cf * Lz);
            } else {
                fy = cf * sy;
                fz = cf * sz;
            }
            R vy[K + 1], vz[K + 1];
#pragma unroll
            for (int r = 0; r <= K; ++r) {
                vy[r] = fy * v[r];
                vz[r] = fz * v[r];
            }
            // a zero factor deposits nothing (a linearly polarised pump keeps A_z = 0)
            if (!wy.put(c - wb, vy)) {
#pragma unroll
                for (int r = 0; r <= K; ++r) atomicAdd(&s_sy[c - r + H], w * (double)vy[r]);
            }
            if (fz != R(0) && !wz.put(c - wb, vz)) {
#pragma unroll
                for (int r = 0; r <= K; ++r) atomicAdd(&s_sz[c - r + H], w * (double)vz[r]);
            }
        }
        tile_release<NS>(Bars, q0 + i);
        if (threadIdx.x == 0 && i + NS < ntile) issue(i + NS);
    }
    if (wb != INT_MIN) {
        wy.flush(s_sy, wb - K + H, w);
        wz.flush(s_sz, wb - K + H, w);
    }
    __syncthreads();
    const bool timeout = *reinterpret_cast<volatile int *>(&Bars.abort) != 0;
    if (timeout && threadIdx.x == 0) {
        atomicOr(A.status, STATUS_TIMEOUT);
        tile_drain<NS>(Bars);
    }
    double *syo = A.s_y, *szo = A.s_z;
    if (A.graph) {                          // replayed by a graph: buffers by sweep parity
        const int it = *reinterpret_cast<volatile const int *>(&A.ctrl->iter);
        syo = A.sypair[it & 1];
        szo = A.szpair[it & 1];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int g = wrap_cell(i - H, A.M);
        const double vy = s_sy[i], vz = s_sz[i];
        if (vy != 0.0) atomicAdd(&syo[g], vy);
        if (vz != 0.0) atomicAdd(&szo[g], vz);
    }
    q = qend;
    return !timeout;
}

template <int K, typename R, int ACC>
__global__ void __launch_bounds__(kSweepThreads, Real<R>::fp32 ? 2 : 1) k_sweep2(Sweep2Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    tile_bars_init(*reinterpret_cast<TileBars *>(smem));
    long long beg, end;
    block_chunk(A.np, beg, end);
    unsigned long long q = 0;
    sweep2_range<K, R, ACC>(A, beg, end, smem, q);
}

size_t sweep2_smem(int M, int H, int fp32)
{
    const size_t W = (size_t)M + 2 * (size_t)H;
    const size_t stages = (size_t)stage_count(fp32) * kTile * (sizeof(int32_t) + 2 * (fp32 ? sizeof(float) : sizeof(double)));
    return 128 + stages + 2 * W * sizeof(double) + (fp32 ? 3 * W * sizeof(float2) : 2 * W * sizeof(double2));
}

// The predicted start's current only sets where the fixed-point iteration starts
// (the fixed point and its stopping test do not depend on it), so its lanes sum in
// the form's own precision: plain float lanes in the FP32 form, whatever
// accumulation the sweeps use.
#define PIC_FOR_PREDEPOSIT_VARIANTS(X)                                                              \
    X(2, double, ACC_NATIVE) X(3, double, ACC_NATIVE) X(4, double, ACC_NATIVE) X(5, double, ACC_NATIVE) \
    X(2, float, ACC_NATIVE) X(3, float, ACC_NATIVE) X(4, float, ACC_NATIVE) X(5, float, ACC_NATIVE)

int launch_predeposit(const Sweep1Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
#define LP(KK, RR, AA)                                                                              \
    if (a.K == KK && (a.fp32 != 0) == std::is_same<RR, float>::value) {                             \
        k_predeposit<KK, RR, AA><<<grid, block, smem, s>>>(a);                                      \
        return 0;                                                                                   \
    }
    PIC_FOR_PREDEPOSIT_VARIANTS(LP)
#undef LP
    return 1;
}

int launch_sweep2(const Sweep2Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
#define L2(KK, RR, AA)                                                                              \
    if (a.K == KK && (a.fp32 != 0) == std::is_same<RR, float>::value && a.acc == AA) {              \
        k_sweep2<KK, RR, AA><<<grid, block, smem, s>>>(a);                                          \
        return 0;                                                                                   \
    }
    PIC_FOR_SWEEP_VARIANTS(L2)
#undef L2
    return 1;
}

// ---------------------------------------------------------------------------
// Diagnostics, evaluated in double from the stored state.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256) k_charge(DiagArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int H = K + 1;
    const int W = A.M + 2 * H;
    double *s_acc = reinterpret_cast<double *>(smem);
    for (int i = threadIdx.x; i < W; i += blockDim.x) s_acc[i] = 0.0;
    __syncthreads();
    const R *tp = static_cast<const R *>(A.P.t);
    // contiguous chunk per block, so a warp's sorted markers share cells: the warp
    // accumulates in a register window (cells wb .. wb+3) and flushes it with
    // shuffles when its lowest cell moves on
    long long beg, end;
    block_chunk(A.np, beg, end);
    DepWindow<double, K + 4, K + 1, K, 0, 3> win;
    win.clear();
    int wb = INT_MIN;
    for (long long a0 = beg; a0 < end; a0 += blockDim.x) {
        const long long a = a0 + threadIdx.x;
        const bool act = a < end;
        const int c = warp_unwrap_cell(act ? A.P.cell[a] : 0, act, A.M, H);   // no reach above
        const int lead = __reduce_min_sync(0xffffffffu, act ? c : INT_MAX);
        if (lead == INT_MAX) break;                    // whole warp past the chunk end
        if (lead != wb) {
            if (wb != INT_MIN) win.advance(lead - wb, s_acc, wb - K + H, A.w);
            wb = lead;
        }
        if (!act) continue;
        double v[K + 1];
        bspline_vals<K, double>((double)tp[a], v);
        if (!win.put(c - wb, v)) {
#pragma unroll
            for (int r = 0; r <= K; ++r) atomicAdd(&s_acc[c - r + H], A.w * v[r]);
        }
    }
    if (wb != INT_MIN) win.flush(s_acc, wb - K + H, A.w);
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const double v = s_acc[i];
        if (v != 0.0) atomicAdd(&A.out[wrap_cell(i - H, A.M)], v);
    }
}

size_t charge_smem(int M, int H) { return ((size_t)M + 2 * (size_t)H) * sizeof(double); }

template <int D, typename R>
__global__ void __launch_bounds__(256) k_gather(DiagArgs A)
{
    const R *tp = static_cast<const R *>(A.P.t);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c = A.P.cell[a];
        double v[D + 1];
        bspline_vals<D, double>((double)tp[a], v);
        double s = 0.0;
#pragma unroll
        for (int r = 0; r <= D; ++r) s += A.c0[wrap_cell(c - r, A.M)] * v[r];
        A.out[A.P.id[a]] = s;
    }
}

template <int K, typename R>
__global__ void __launch_bounds__(256) k_kinetic(DiagArgs A)
{
    __shared__ double s_red[32];
    const R *tp = static_cast<const R *>(A.P.t);
    const R *pp = static_cast<const R *>(A.P.p);
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c = A.P.cell[a];
        double v[K + 1];
        bspline_vals<K, double>((double)tp[a], v);
        double Ay = 0.0, Az = 0.0;
#pragma unroll
        for (int r = 0; r <= K; ++r) {
            const int i = wrap_cell(c - r, A.M);
            Ay += A.c0[i] * v[r];
            Az += A.c1[i] * v[r];
        }
        const double p = (double)pp[a];
        const double q = p * p + Ay * Ay + Az * Az;
        acc += A.w * q / (1.0 + sqrt(1.0 + q));      // w (gamma - 1) without cancellation
    }
    block_sum_to(A.acc, acc, s_red);
}

template <typename R>
static int launch_charge_t(const DiagArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    switch (a.K) {
    case 2: k_charge<2, R><<<grid, block, smem, s>>>(a); break;
    case 3: k_charge<3, R><<<grid, block, smem, s>>>(a); break;
    case 4: k_charge<4, R><<<grid, block, smem, s>>>(a); break;
    case 5: k_charge<5, R><<<grid, block, smem, s>>>(a); break;
    default: return 1;
    }
    return 0;
}

int launch_charge(const DiagArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    return a.fp32 ? launch_charge_t<float>(a, grid, block, smem, s)
                  : launch_charge_t<double>(a, grid, block, smem, s);
}

template <typename R>
static int launch_gather_t(const DiagArgs &a, int d, int grid, int block, cudaStream_t s)
{
    switch (d) {
    case 1: k_gather<1, R><<<grid, block, 0, s>>>(a); break;
    case 2: k_gather<2, R><<<grid, block, 0, s>>>(a); break;
    case 3: k_gather<3, R><<<grid, block, 0, s>>>(a); break;
    case 4: k_gather<4, R><<<grid, block, 0, s>>>(a); break;
    case 5: k_gather<5, R><<<grid, block, 0, s>>>(a); break;
    default: return 1;
    }
    return 0;
}

int launch_gather(const DiagArgs &a, int d, int grid, int block, cudaStream_t s)
{
    return a.fp32 ? launch_gather_t<float>(a, d, grid, block, s)
                  : launch_gather_t<double>(a, d, grid, block, s);
}

// Path mean of E_x,h = sum_i e_i Lambda^1_i along x_a -> x_a + d_a (Sec. 4.2, the
// (1/dt) int Lambda_1(X(tau)) dtau . e of subsystem I), in double: the path is
// split at the knots and each piece contributes (h/d) times the exact means of
// the degree-(K-1) pieces; a zero displacement gives E_x,h(x_a).  On entry
// out[id] holds d (length units); it is overwritten with the mean.
template <int K, typename R>
__global__ void __launch_bounds__(256) k_gather_path(DiagArgs A)
{
    const R *tp = static_cast<const R *>(A.P.t);
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c0 = A.P.cell[a];
        const int id = A.P.id[a];
        const double d = A.out[id] / A.dx;
        if (!(fabs(d) <= (double)A.Dlim)) { bad = true; A.out[id] = 0.0; continue; }
        double mean = 0.0;
        const double invd = d != 0.0 ? 1.0 / d : 0.0;
        walk_path<K, double>((double)tp[a], d, [&](int c, double h, const double *m, bool single) {
            double e = 0.0;
#pragma unroll
            for (int r = 0; r < K; ++r) e += m[r] * A.c0[wrap_cell(c0 + c - r, A.M)];
            mean += single ? e : h * invd * e;
        });
        A.out[id] = mean;
    }
    if (bad) atomicOr(A.status, STATUS_NUMERIC);
}

// ---------------------------------------------------------------------------
// Spin (double form): deposit, rotation (subsystem III) and Zeeman energy.  Spin
// components live in caller order; markers are visited in stored order and
// their spins addressed through id.
// ---------------------------------------------------------------------------
// dA/dx at a marker: sum_i (G a)_i Lambda^1_i(x), (G a)_i = (a_i - a_{i-1}) / dx
template <int K>
__device__ __forceinline__ void spin_field_grad(const SpinArgs &A, int c, double t, double &Y, double &Z)
{
    double v[K];
    bspline_vals<K - 1, double>(t, v);
    Y = 0.0;
    Z = 0.0;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int i = wrap_cell(c - r, A.M), im = wrap_cell(c - r - 1, A.M);
        Y += v[r] * (A.ay[i] - A.ay[im]);
        Z += v[r] * (A.az[i] - A.az[im]);
    }
    Y /= A.dx;
    Z /= A.dx;
}

template <int K>
__global__ void __launch_bounds__(256) k_spin_deposit(SpinArgs A)
{
    extern __shared__ __align__(16) double s_dep[];
    double *sy = s_dep, *sz = s_dep + A.M;
    for (int i = threadIdx.x; i < 2 * A.M; i += blockDim.x) s_dep[i] = 0.0;
    __syncthreads();
    const double *tp = static_cast<const double *>(A.P.t);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c = A.P.cell[a];
        const int id = A.P.id[a];
        double v[K];
        bspline_vals<K - 1, double>(tp[a], v);
        const double wy = A.w * A.sy[id], wz = A.w * A.sz[id];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = wrap_cell(c - r, A.M);
            atomicAdd(&sy[i], wy * v[r]);
            atomicAdd(&sz[i], wz * v[r]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < A.M; i += blockDim.x) {
        if (sy[i] != 0.0) atomicAdd(&A.dy[i], sy[i]);
        if (sz[i] != 0.0) atomicAdd(&A.dz[i], sz[i]);
    }
}

// Subsystem III (Eq. spin_rodrigue): s <- s + sin(dt|r|)/|r| (r x s)
//                                         + (1/2) (sin(dt|r|/2)/(|r|/2))^2 r x (r x s),
// r = (0, Z, -Y), Y = dA_y/dx, Z = dA_z/dx at the marker.
template <int K>
__global__ void __launch_bounds__(256) k_spin_rotate(SpinArgs A)
{
    const double *tp = static_cast<const double *>(A.P.t);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int id = A.P.id[a];
        double Y, Z;
        spin_field_grad<K>(A, A.P.cell[a], tp[a], Y, Z);
        const double r1 = Z, r2 = -Y;
        const double nr = sqrt(r1 * r1 + r2 * r2);
        const double s0 = A.sx[id], s1 = A.sy[id], s2 = A.sz[id];
        // c1 = r x s, c2 = r x c1, with r0 = 0
        const double c1x = r1 * s2 - r2 * s1, c1y = r2 * s0, c1z = -r1 * s0;
        const double c2x = r1 * c1z - r2 * c1y, c2y = r2 * c1x, c2z = -r1 * c1x;
        double f1, f2;
        if (nr > 0.0) {
            f1 = sin(A.dt * nr) / nr;
            const double hh = sin(0.5 * A.dt * nr) / (0.5 * nr);
            f2 = 0.5 * hh * hh;
        } else {
            f1 = A.dt;
            f2 = 0.5 * A.dt * A.dt;
        }
        A.sx[id] = s0 + f1 * c1x + f2 * c2x;
        A.sy[id] = s1 + f1 * c1y + f2 * c2y;
        A.sz[id] = s2 + f1 * c1z + f2 * c2z;
    }
}

template <int K>
__global__ void __launch_bounds__(256) k_spin_energy(SpinArgs A)
{
    __shared__ double s_red[32];
    const double *tp = static_cast<const double *>(A.P.t);
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int id = A.P.id[a];
        double Y, Z;
        spin_field_grad<K>(A, A.P.cell[a], tp[a], Y, Z);
        acc += A.w * (A.sy[id] * Z - A.sz[id] * Y);
    }
    block_sum_to(A.acc, acc, s_red);
}

#define PIC_SPIN_LAUNCH(NAME, SMEM)                                                      \
    switch (a.K) {                                                                       \
    case 2: NAME<2><<<grid, 256, SMEM, s>>>(a); break;                                   \
    case 3: NAME<3><<<grid, 256, SMEM, s>>>(a); break;                                   \
    case 4: NAME<4><<<grid, 256, SMEM, s>>>(a); break;                                   \
    case 5: NAME<5><<<grid, 256, SMEM, s>>>(a); break;                                   \
    default: return 1;                                                                   \
    }                                                                                    \
    return 0;

int launch_spin_deposit(const SpinArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = 2 * (size_t)a.M * sizeof(double);
    PIC_SPIN_LAUNCH(k_spin_deposit, smem)
}

int launch_spin_rotate(const SpinArgs &a, int grid, cudaStream_t s) { PIC_SPIN_LAUNCH(k_spin_rotate, 0) }

int launch_spin_energy(const SpinArgs &a, int grid, cudaStream_t s) { PIC_SPIN_LAUNCH(k_spin_energy, 0) }

#undef PIC_SPIN_LAUNCH

int launch_gather_path(const DiagArgs &a, int grid, int block, cudaStream_t s)
{
#define GP(KK)                                                                                  \
    case KK:                                                                                    \
        if (a.fp32) k_gather_path<KK, float><<<grid, block, 0, s>>>(a);                         \
        else k_gather_path<KK, double><<<grid, block, 0, s>>>(a);                               \
        break;
    switch (a.K) {
    GP(2) GP(3) GP(4) GP(5)
    default: return 1;
    }
#undef GP
    return 0;
}

template <typename R>
static int launch_kinetic_t(const DiagArgs &a, int grid, int block, cudaStream_t s)
{
    switch (a.K) {
    case 2: k_kinetic<2, R><<<grid, block, 0, s>>>(a); break;
    case 3: k_kinetic<3, R><<<grid, block, 0, s>>>(a); break;
    case 4: k_kinetic<4, R><<<grid, block, 0, s>>>(a); break;
    case 5: k_kinetic<5, R><<<grid, block, 0, s>>>(a); break;
    default: return 1;
    }
    return 0;
}

int launch_kinetic(const DiagArgs &a, int grid, int block, cudaStream_t s)
{
    return a.fp32 ? launch_kinetic_t<float>(a, grid, block, s)
                  : launch_kinetic_t<double>(a, grid, block, s);
}

// ---------------------------------------------------------------------------
// End of subsystem I: x^{n+1} = x^n + delta (re-split into cell and offset,
// wrapped periodically), p^{n+1} = p^(k+1).  delta is cleared only where the
// next iteration starts from it (no warm start): the warm starts overwrite it
// before any sweep reads it.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void finalize1_range(long long np, int M, const PartPtrs &P, long long a0,
                                                long long stride, bool zero_delta)
{
    R *tp = static_cast<R *>(P.t);
    R *pp = static_cast<R *>(P.p);
    R *dp = static_cast<R *>(P.delta);
    const R *pnp = static_cast<const R *>(P.pnew);
    for (long long a = a0; a < np; a += stride) {
        const R s = tp[a] + dp[a];
        const R f = floor_(s);
        int c = P.cell[a] + (int)f;
        R t = s - f;
        if (t >= R(1)) { t -= R(1); c += 1; }
        P.cell[a] = wrap_cell(c, M);
        tp[a] = t;
        pp[a] = pnp[a];
        if (zero_delta) dp[a] = R(0);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_finalize1(long long np, int M, PartPtrs P, bool zero_delta)
{
    finalize1_range<R>(np, M, P, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                       (long long)gridDim.x * blockDim.x, zero_delta);
}

int launch_finalize1(int fp32, long long np, int M, PartPtrs P, bool zero_delta, int grid, int block,
                     cudaStream_t s)
{
    if (fp32) k_finalize1<float><<<grid, block, 0, s>>>(np, M, P, zero_delta);
    else k_finalize1<double><<<grid, block, 0, s>>>(np, M, P, zero_delta);
    return 0;
}

// ---------------------------------------------------------------------------
// Load / store between the caller's FP64 (x, p) arrays and the stored form.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_load(long long np, int M, double dx, const double *x,
                                              const double *p, PartPtrs P)
{
    R *tp = static_cast<R *>(P.t);
    R *pp = static_cast<R *>(P.p);
    R *dp = static_cast<R *>(P.delta);
    R *pnp = static_cast<R *>(P.pnew);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < np; a += stride) {
        const double u = x[a] / dx;
        const double f = ::floor(u);
        int c = (int)f;
        R t = (R)(u - f);
        if (t >= R(1)) { t = R(0); c += 1; }
        P.cell[a] = wrap_cell(c, M);
        tp[a] = t;
        pp[a] = (R)p[a];
        pnp[a] = (R)p[a];
        dp[a] = R(0);
        P.id[a] = (int32_t)a;
    }
}

int launch_load(int fp32, long long np, int M, double dx, const double *x, const double *p,
                PartPtrs P, int grid, int block, cudaStream_t s)
{
    if (fp32) k_load<float><<<grid, block, 0, s>>>(np, M, dx, x, p, P);
    else k_load<double><<<grid, block, 0, s>>>(np, M, dx, x, p, P);
    return 0;
}

template <typename R>
__global__ void __launch_bounds__(256) k_store(long long np, double dx, PartPtrs P, double *x, double *p)
{
    const R *tp = static_cast<const R *>(P.t);
    const R *pp = static_cast<const R *>(P.p);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < np; a += stride) {
        const long long i = P.id[a];
        if (x) x[i] = ((double)P.cell[a] + (double)tp[a]) * dx;
        if (p) p[i] = (double)pp[a];
    }
}

int launch_store(int fp32, long long np, double dx, PartPtrs P, double *x, double *p,
                 int grid, int block, cudaStream_t s)
{
    if (fp32) k_store<float><<<grid, block, 0, s>>>(np, dx, P, x, p);
    else k_store<double><<<grid, block, 0, s>>>(np, dx, P, x, p);
    return 0;
}

// inv[id[a]] = a: where the marker of each caller index is stored
__global__ void __launch_bounds__(256) k_inverse_id(long long np, const int32_t *__restrict__ id,
                                                    int32_t *__restrict__ inv)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < np; a += stride)
        inv[id[a]] = (int32_t)a;
}

// x[i], p[i] in caller order, each read from where marker i is stored: the writes are
// consecutive, so the destination may be page-locked host memory written over the host
// link (the same values as k_store)
template <typename R>
__global__ void __launch_bounds__(256) k_store_ordered(long long np, double dx, PartPtrs P,
                                                       const int32_t *__restrict__ inv, double *x, double *p)
{
    const R *tp = static_cast<const R *>(P.t);
    const R *pp = static_cast<const R *>(P.p);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
        const long long a = inv[i];
        if (x) x[i] = ((double)P.cell[a] + (double)tp[a]) * dx;
        if (p) p[i] = (double)pp[a];
    }
}

int launch_store_ordered(int fp32, long long np, double dx, PartPtrs P, int32_t *inv, double *x, double *p,
                         int grid, int block, cudaStream_t s)
{
    k_inverse_id<<<grid, block, 0, s>>>(np, P.id, inv);
    if (fp32) k_store_ordered<float><<<grid, block, 0, s>>>(np, dx, P, inv, x, p);
    else k_store_ordered<double><<<grid, block, 0, s>>>(np, dx, P, inv, x, p);
    return 0;
}

// ---------------------------------------------------------------------------
// Counting sort of the markers by key = cell * nbins + velocity bin, the bin being
// the expected displacement tau p in units of 1/per cell (nbins = 16 per, clamped),
// so that a warp's markers share cells and piece counts.  Runs between steps; delta and
// p_new are not carried (each step's first sweep or warm start writes them
// before they are read, and delta is all zero where the iteration starts from
// it).  Atomics are aggregated per warp over equal keys.
// counts: 2 * nkeys int32 (histogram, then cursors).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int sort_key(int c, R p, float taup, int nbins)
{
    int b = (int)floorf((float)p * taup) + nbins / 2;
    b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
    return c * nbins + b;
}

// Both passes give each block a contiguous chunk of the markers.  The markers are
// nearly sorted (they were sorted a few steps ago), so the blocks running at the
// same time then touch different keys' counters; in a grid-stride order every
// block would work on the same few cells at once and serialise on their counters.
// chunk [beg, end) of block b among nb blocks (a multiple of 32 markers)
__device__ __forceinline__ void chunk_of(long long np, int b, int nb, long long &beg, long long &end)
{
    long long chunk = (np + nb - 1) / nb;
    chunk = (chunk + 31) & ~31LL;
    beg = (long long)b * chunk;
    end = beg + chunk < np ? beg + chunk : np;
}

template <typename R>
__device__ __forceinline__ void hist_range(long long beg, long long end, float tau, int nbins, const PartPtrs &S,
                                           int32_t *counts)
{
    const R *ps = static_cast<const R *>(S.p);
    const int lane = threadIdx.x & 31;
    for (long long base = beg; base < end; base += blockDim.x) {
        const long long a = base + threadIdx.x;
        const bool act = a < end;
        const int key = act ? sort_key(S.cell[a], ps[a], tau, nbins) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (act && lane == __ffs(grp) - 1) atomicAdd(&counts[key], __popc(grp));
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_hist(long long np, float tau, int nbins, PartPtrs S, int32_t *counts)
{
    long long beg, end;
    block_chunk(np, beg, end);
    hist_range<R>(beg, end, tau, nbins, S, counts);
}

__device__ __forceinline__ void scan_block(int nkeys, int32_t *counts)
{
    // exclusive scan of nkeys counts into cursors (single block)
    __shared__ int s_part[1024];
    const int per = (nkeys + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(nkeys, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    s_part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int v = threadIdx.x >= (unsigned)off ? s_part[threadIdx.x - off] : 0;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = s_part[threadIdx.x] - s;     // exclusive prefix of this thread's range
    for (int i = lo; i < hi; ++i) { const int v = counts[i]; counts[nkeys + i] = run; run += v; }
}

__global__ void __launch_bounds__(1024) k_scan(int nkeys, int32_t *counts) { scan_block(nkeys, counts); }

template <typename R>
__device__ __forceinline__ void scatter_range(long long beg, long long end, float tau, int nbins, const PartPtrs &S,
                                              const PartPtrs &D, int32_t *cursor)
{
    const R *ts = static_cast<const R *>(S.t);
    const R *ps = static_cast<const R *>(S.p);
    R *td = static_cast<R *>(D.t);
    R *pd = static_cast<R *>(D.p);
    const int lane = threadIdx.x & 31;
    // kSortU markers a thread per pass: their cursor atomics are independent, so
    // the warp waits for the returned slots once per pass instead of once a marker
    constexpr int kSortU = 4;
    for (long long base = beg; base < end; base += kSortU * (long long)blockDim.x) {
        int c[kSortU], key[kSortU], first[kSortU];
        R p[kSortU];
        unsigned grp[kSortU];
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            const long long a = base + u * (long long)blockDim.x + threadIdx.x;
            const bool act = a < end;
            c[u] = act ? S.cell[a] : 0;
            p[u] = act ? ps[a] : R(0);
            key[u] = act ? sort_key(c[u], p[u], tau, nbins) : -1;
        }
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            grp[u] = __match_any_sync(0xffffffffu, key[u]);
            first[u] = 0;
            if (key[u] >= 0 && lane == __ffs(grp[u]) - 1) first[u] = atomicAdd(&cursor[key[u]], __popc(grp[u]));
        }
#pragma unroll
        for (int u = 0; u < kSortU; ++u) {
            const long long a = base + u * (long long)blockDim.x + threadIdx.x;
            const int f = __shfl_sync(0xffffffffu, first[u], __ffs(grp[u]) - 1);
            if (key[u] < 0) continue;
            const long long j = (long long)f + __popc(grp[u] & ((1u << lane) - 1u));
            D.cell[j] = c[u];
            td[j] = ts[a];
            pd[j] = p[u];
            D.id[j] = S.id[a];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_scatter(long long np, float tau, int nbins, PartPtrs S, PartPtrs D,
                                                 int32_t *cursor)
{
    long long beg, end;
    block_chunk(np, beg, end);
    scatter_range<R>(beg, end, tau, nbins, S, D, cursor);
}

// Batched sorts (ensembles): block row y = run, its counts zeroed, histogrammed,
// scanned (one block a run) and scattered in four launches for all runs due.
__global__ void __launch_bounds__(256) k_sort_zero_ens(const SortRun *runs)
{
    const SortRun &r = runs[blockIdx.y];
    const int n = 2 * r.M * r.nbins;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r.counts[i] = 0;
}

template <typename R>
__global__ void __launch_bounds__(256) k_hist_ens(const SortRun *runs)
{
    const SortRun &r = runs[blockIdx.y];
    long long beg, end;
    chunk_of(r.np, blockIdx.x, gridDim.x, beg, end);
    hist_range<R>(beg, end, r.taup, r.nbins, r.src, r.counts);
}

__global__ void __launch_bounds__(1024) k_scan_ens(const SortRun *runs)
{
    const SortRun &r = runs[blockIdx.x];
    scan_block(r.M * r.nbins, r.counts);
}

template <typename R>
__global__ void __launch_bounds__(256) k_scatter_ens(const SortRun *runs)
{
    const SortRun &r = runs[blockIdx.y];
    long long beg, end;
    chunk_of(r.np, blockIdx.x, gridDim.x, beg, end);
    scatter_range<R>(beg, end, r.taup, r.nbins, r.src, r.dst, r.counts + (size_t)r.M * r.nbins);
}

int launch_sort_ens(int fp32, const SortRun *runs, int nruns, int grid_x, cudaStream_t s)
{
    if (nruns < 1) return 0;
    const dim3 g(grid_x, nruns);
    k_sort_zero_ens<<<g, 256, 0, s>>>(runs);
    if (fp32) k_hist_ens<float><<<g, 256, 0, s>>>(runs);
    else k_hist_ens<double><<<g, 256, 0, s>>>(runs);
    k_scan_ens<<<nruns, 1024, 0, s>>>(runs);
    if (fp32) k_scatter_ens<float><<<g, 256, 0, s>>>(runs);
    else k_scatter_ens<double><<<g, 256, 0, s>>>(runs);
    return 0;
}

int launch_sort(int fp32, long long np, int M, double tau, int per, PartPtrs src, PartPtrs dst,
                int32_t *counts, int grid, int block, cudaStream_t s)
{
    const int nbins = kVelBinsBase * per;
    const int nkeys = M * nbins;
    const float taup = (float)(tau * per);
    if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * (size_t)nkeys, s) != cudaSuccess) return 1;
    if (fp32) k_hist<float><<<grid, block, 0, s>>>(np, taup, nbins, src, counts);
    else k_hist<double><<<grid, block, 0, s>>>(np, taup, nbins, src, counts);
    k_scan<<<1, 1024, 0, s>>>(nkeys, counts);
    if (fp32) k_scatter<float><<<grid, block, 0, s>>>(np, taup, nbins, src, dst, counts + nkeys);
    else k_scatter<double><<<grid, block, 0, s>>>(np, taup, nbins, src, dst, counts + nkeys);
    return 0;
}

// ---------------------------------------------------------------------------
// Dynamic shared-memory opt-in (per kernel instantiation) and occupancy.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Batched ensemble sweeps: persistent blocks claim work items (run, marker range)
// until the queue built by the plan kernel is empty.  Item boundaries are
// multiples of the tile size, so every bulk copy stays 16-byte aligned.  After a
// bounded wait gave up (the run's status records it) the block stops claiming.
// ---------------------------------------------------------------------------
template <typename Args>
__device__ __forceinline__ bool ens_claim(EnsQueue *Q, const Args *runs, int nruns, int &run,
                                          long long &beg, long long &end)
{
    __shared__ int s_item;
    __syncthreads();                       // s_item of the previous claim is consumed
    if (threadIdx.x == 0) s_item = atomicAdd(&Q->next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= Q->nitems) return false;
    // the run r with item_start[r] <= item < item_start[r + 1]
    int lo = 0, hi = nruns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (Q->item_start[mid] <= item) lo = mid; else hi = mid;
    }
    run = lo;
    const long long im = Q->item_markers;
    beg = (long long)(item - Q->item_start[run]) * im;
    end = beg + im < runs[run].np ? beg + im : runs[run].np;
    return true;
}

template <int K, typename R>
__global__ void __launch_bounds__(kSweepThreads, Real<R>::fp32 ? 2 : 1)
    k_sweep1_ens(const Sweep1Args *runs, int nruns, EnsQueue *Q)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if ((int)blockIdx.x >= Q->nblocks) return;
    tile_bars_init(*reinterpret_cast<TileBars *>(smem));
    unsigned long long q = 0;
    int run;
    long long beg, end;
    while (ens_claim(Q, runs, nruns, run, beg, end))
        if (!sweep1_range<K, R, DefaultAcc<R>::v>(runs[run], beg, end, smem, q)) break;
}

// the predicted start of every run (sweep1_range's PRE mode over the work queue)
template <int K, typename R>
__global__ void __launch_bounds__(kSweepThreads, Real<R>::fp32 ? 2 : 1)
    k_predeposit_ens(const Sweep1Args *runs, int nruns, EnsQueue *Q)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if ((int)blockIdx.x >= Q->nblocks) return;
    tile_bars_init(*reinterpret_cast<TileBars *>(smem));
    unsigned long long q = 0;
    int run;
    long long beg, end;
    while (ens_claim(Q, runs, nruns, run, beg, end))
        if (!sweep1_range<K, R, ACC_NATIVE, true>(runs[run], beg, end, smem, q)) break;
}

template <int K, typename R>
__global__ void __launch_bounds__(kSweepThreads, Real<R>::fp32 ? 2 : 1)
    k_sweep2_ens(const Sweep2Args *runs, int nruns, EnsQueue *Q)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if ((int)blockIdx.x >= Q->nblocks) return;
    tile_bars_init(*reinterpret_cast<TileBars *>(smem));
    unsigned long long q = 0;
    int run;
    long long beg, end;
    while (ens_claim(Q, runs, nruns, run, beg, end))
        if (!sweep2_range<K, R, DefaultAcc<R>::v>(runs[run], beg, end, smem, q)) break;
}

template <typename R>
static int launch_sweep_ens_t(int which, int K, const void *runs, int nruns, EnsQueue *Q, int grid,
                              size_t smem, cudaStream_t s)
{
    const int b = kSweepThreads;
#define ENS(KK)                                                                                          \
    case KK:                                                                                             \
        if (which == 1) k_sweep1_ens<KK, R><<<grid, b, smem, s>>>((const Sweep1Args *)runs, nruns, Q);   \
        else if (which == 2) k_sweep2_ens<KK, R><<<grid, b, smem, s>>>((const Sweep2Args *)runs, nruns, Q); \
        else k_predeposit_ens<KK, R><<<grid, b, smem, s>>>((const Sweep1Args *)runs, nruns, Q);        \
        break;
    switch (K) {
    ENS(2) ENS(3) ENS(4) ENS(5)
    default: return 1;
    }
#undef ENS
    return 0;
}

int launch_sweep1_ens(int K, int fp32, const Sweep1Args *runs, int nruns, EnsQueue *Q, int grid,
                      size_t smem, cudaStream_t s)
{
    return fp32 ? launch_sweep_ens_t<float>(1, K, runs, nruns, Q, grid, smem, s)
                : launch_sweep_ens_t<double>(1, K, runs, nruns, Q, grid, smem, s);
}

int launch_sweep2_ens(int K, int fp32, const Sweep2Args *runs, int nruns, EnsQueue *Q, int grid,
                      size_t smem, cudaStream_t s)
{
    return fp32 ? launch_sweep_ens_t<float>(2, K, runs, nruns, Q, grid, smem, s)
                : launch_sweep_ens_t<double>(2, K, runs, nruns, Q, grid, smem, s);
}

int launch_predeposit_ens(int K, int fp32, const Sweep1Args *runs, int nruns, EnsQueue *Q, int grid,
                          size_t smem, cudaStream_t s)
{
    return fp32 ? launch_sweep_ens_t<float>(0, K, runs, nruns, Q, grid, smem, s)
                : launch_sweep_ens_t<double>(0, K, runs, nruns, Q, grid, smem, s);
}

// End of subsystem I for every run (block row = run); runs stopped by an error
// keep their markers.
template <typename R>
__global__ void __launch_bounds__(256) k_finalize1_ens(const RunDesc *runs)
{
    const RunDesc &D = runs[blockIdx.y];
    if (D.ctrl->status & (STATUS_NUMERIC | STATUS_TIMEOUT)) return;
    finalize1_range<R>(D.np, D.M, D.P, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                       (long long)gridDim.x * blockDim.x, true);
}

int launch_finalize1_ens(int fp32, const RunDesc *R, int nruns, int grid_x, cudaStream_t s)
{
    if (fp32) k_finalize1_ens<float><<<dim3(grid_x, nruns), 256, 0, s>>>(R);
    else k_finalize1_ens<double><<<dim3(grid_x, nruns), 256, 0, s>>>(R);
    return 0;
}

template <int K, typename R>
static int set_attrs_kr(size_t s1, size_t s2, size_t s3)
{
    if (cudaFuncSetAttribute(k_sweep1_ens<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) return 1;
    if (cudaFuncSetAttribute(k_predeposit_ens<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) return 1;
    if (cudaFuncSetAttribute(k_sweep2_ens<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2)) return 1;
    if (cudaFuncSetAttribute(k_current<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3)) return 1;
    if (cudaFuncSetAttribute(k_charge<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3)) return 1;
    return 0;
}

template <typename R>
static int set_attrs_r(size_t s1, size_t s2, size_t s3)
{
    return set_attrs_kr<2, R>(s1, s2, s3) | set_attrs_kr<3, R>(s1, s2, s3) |
           set_attrs_kr<4, R>(s1, s2, s3) | set_attrs_kr<5, R>(s1, s2, s3);
}

static int set_attrs_sweeps(size_t s1, size_t s2, size_t s3)
{
    int rc = 0;
#define ATTRV(KK, RR, AA)                                                                               \
    rc |= cudaFuncSetAttribute(k_sweep1<KK, RR, AA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1) != \
          cudaSuccess;                                                                                  \
    rc |= cudaFuncSetAttribute(k_sweep2<KK, RR, AA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2) != \
          cudaSuccess;
    PIC_FOR_SWEEP_VARIANTS(ATTRV)
#undef ATTRV
#define ATTRP(KK, RR, AA)                                                                               \
    rc |= cudaFuncSetAttribute(k_predeposit<KK, RR, AA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1) != \
          cudaSuccess;
    PIC_FOR_PREDEPOSIT_VARIANTS(ATTRP)
#undef ATTRP
    return rc;
}

static int set_attrs_spin(size_t smem)
{
    int rc = 0;
    rc |= cudaFuncSetAttribute(k_spin_deposit<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess;
    rc |= cudaFuncSetAttribute(k_spin_deposit<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess;
    rc |= cudaFuncSetAttribute(k_spin_deposit<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess;
    rc |= cudaFuncSetAttribute(k_spin_deposit<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess;
    return rc;
}

int spin_optin(int M)
{
    static std::mutex mu;
    static size_t have = 0;
    std::lock_guard<std::mutex> lock(mu);
    const size_t need = 2 * (size_t)M * sizeof(double);
    if (need <= have) return 0;
    if (set_attrs_spin(need)) return 1;
    have = need;
    return 0;
}

int sweep_blocks_per_sm(int K, int fp32, int acc, int which, int block, size_t smem)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define OCC(KK, RR, AA)                                                                                   \
    if (K == KK && (fp32 != 0) == std::is_same<RR, float>::value && acc == AA)                           \
        e = which == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep1<KK, RR, AA>, block, smem) \
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<KK, RR, AA>, block, smem);
    PIC_FOR_SWEEP_VARIANTS(OCC)
#undef OCC
    return e == cudaSuccess ? n : 0;
}

}  // namespace pic

// Raises the dynamic shared-memory limits of the marker kernels to at least
// (s1, s2, s3) bytes; never lowers them, so handles of different grid sizes can
// coexist in one process.
int pic_set_smem_attrs(size_t s1, size_t s2, size_t s3)
{
    static std::mutex mu;
    static size_t m1 = 0, m2 = 0, m3 = 0;
    std::lock_guard<std::mutex> lock(mu);
    const size_t n1 = std::max(m1, s1), n2 = std::max(m2, s2), n3 = std::max(m3, s3);
    if (n1 == m1 && n2 == m2 && n3 == m3) return 0;
    const int rc = pic::set_attrs_r<float>(n1, n2, n3) | pic::set_attrs_r<double>(n1, n2, n3) |
                   pic::set_attrs_sweeps(n1, n2, n3);
    if (rc == 0) { m1 = n1; m2 = n2; m3 = n3; }
    return rc;
}
