// pic_device.cuh -- device-side building blocks of libpic (sm_103a).
//
// Positions are stored as (cell c, offset t in [0,1)) in cell units: x = (c + t) dx.
// In cell c the degree-d periodic basis functions j = c - r (r = 0..d) are nonzero
// with values N^d(r + t), N^d the cardinal B-spline on the integer knots (Sec. 3.1:
// Lambda^0_j = N^k_j, Lambda^1_j = N^{k-1}_j, supp N^d_j = [x_j, x_{j+d+1})).
#pragma once

#include <climits>
#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

// ---------------------------------------------------------------------------
// Device control block of one fixed-point loop.
// Non-negative doubles are kept as their bit patterns so that integer atomicMax
// orders them; NaN (0x7ff8...) compares above +Inf, so it reads "not converged".
// ---------------------------------------------------------------------------
struct DevCtrl {
    unsigned long long dmax_bits;      // max particle increment of this sweep
    unsigned long long emax_bits;      // max field increment of this sweep
    unsigned long long dprev_bits;     // previous sweep's values (stagnation test)
    unsigned long long eprev_bits;
    unsigned long long emag_bits;      // max |e^(k+1)| of this sweep (field scale)
    int iter;                          // sweeps done in the current loop
    int converged;                     // 1 once the test passed
    int status;                        // error bits, see STATUS_*
    unsigned int ticket;               // last-block election in multi-block grid kernels
    int hist1, hist2;                  // field changes stored for the starting fields
    double acc[4];                     // reductions for diagnostics (energy, residual)
};

enum : int {
    STATUS_NUMERIC = 1,    // NaN/Inf or displacement beyond the halo
    STATUS_NOCONV  = 2,
    STATUS_TIMEOUT = 4,    // a bounded wait on a bulk copy gave up
};

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the TMA engine's 1-D bulk mode) into shared memory,
// completed on an mbarrier.  Every wait is bounded: after kMaxWaitTries polls it
// returns false and the caller records STATUS_TIMEOUT and leaves.  Addresses and
// sizes must be multiples of 16 bytes.
// ---------------------------------------------------------------------------
constexpr unsigned long long kMaxWaitTries = 1ull << 26;

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// one arrival (release semantics: this thread's earlier shared-memory reads are
// ordered before the barrier's phase completes)
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (unsigned long long i = 0; i < kMaxWaitTries; ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v)
{
    // v >= 0 or NaN: the IEEE bit pattern is monotone in v for non-negative values
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double bits_to_double(unsigned long long b)
{
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ int wrap_cell(int c, int M)
{
    c %= M;
    return c < 0 ? c + M : c;
}

template <typename R> __device__ __forceinline__ R rsqrt_(R v);
template <> __device__ __forceinline__ float rsqrt_(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ double rsqrt_(double v) { return rsqrt(v); }

template <typename R> __device__ __forceinline__ R sqrt_(R v);
template <> __device__ __forceinline__ float sqrt_(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }

template <typename R> __device__ __forceinline__ R floor_(R v);
template <> __device__ __forceinline__ float floor_(float v) { return floorf(v); }
template <> __device__ __forceinline__ double floor_(double v) { return ::floor(v); }

// ---------------------------------------------------------------------------
// Uniform B-spline values by the triangular (de Boor) scheme:
// level 0: b = [1]; level n: b'_r = ((t + r) b_r + (n + 1 - t - r) b_{r-1}) / n,
// with b_{-1} = b_n = 0.  After level d, v[r] = N^d(r + t), r = 0..d.
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void bspline_vals(R t, R *v)
{
    v[0] = R(1);
#pragma unroll
    for (int n = 1; n <= D; ++n) {
        const R inv = R(1) / R(n);
        v[n] = (R(1) - t) * v[n - 1] * inv;
#pragma unroll
        for (int r = n - 1; r >= 1; --r)
            v[r] = ((t + R(r)) * v[r] + (R(n + 1 - r) - t) * v[r - 1]) * inv;
        v[0] = t * v[0] * inv;
    }
}

// Same triangle, also returning the level D-2 and D-4 values (second and fourth
// derivatives of the pieces by the derivative relation of Sec. 3.1 applied twice:
// d^2/ds^2 N^D(s) = N^{D-2}(s) - 2 N^{D-2}(s-1) + N^{D-2}(s-2)).
template <int D, typename R>
__device__ __forceinline__ void bspline_vals_levels(R t, R *v, R *lv2, R *lv4)
{
    v[0] = R(1);
    if (D == 2) lv2[0] = R(1);
    if (D == 4) lv4[0] = R(1);
#pragma unroll
    for (int n = 1; n <= D; ++n) {
        const R inv = R(1) / R(n);
        v[n] = (R(1) - t) * v[n - 1] * inv;
#pragma unroll
        for (int r = n - 1; r >= 1; --r)
            v[r] = ((t + R(r)) * v[r] + (R(n + 1 - r) - t) * v[r - 1]) * inv;
        v[0] = t * v[0] * inv;
        if (n == D - 2) {
#pragma unroll
            for (int r = 0; r <= (D - 2 > 0 ? D - 2 : 0); ++r) lv2[r] = v[r];
        }
        if (n == D - 4) {
#pragma unroll
            for (int r = 0; r <= (D - 4 > 0 ? D - 4 : 0); ++r) lv4[r] = v[r];
        }
    }
}

// Mean of the D+1 pieces N^D(r + t), r = 0..D, over the local interval centred at
// tm with signed length h (|h| <= 1), exact for polynomials of degree <= 5:
//   mean f = f(tm) + f''(tm) h^2 / 24 + f''''(tm) h^4 / 1920.
// (Midpoint Taylor expansion of the interval mean; odd terms cancel.)
template <int D, typename R>
__device__ __forceinline__ void piece_means(R tm, R h, R *m)
{
    static_assert(D >= 0 && D <= 5, "degree");
    if (D < 2) {
        bspline_vals<D, R>(tm, m);
        return;
    }
    R l2[D + 1 > 1 ? D + 1 : 1];
    R l4[D + 1 > 1 ? D + 1 : 1];
    bspline_vals_levels<D, R>(tm, m, l2, l4);
    const R h2 = h * h * R(1.0 / 24.0);
#pragma unroll
    for (int r = 0; r <= D; ++r) {
        // second difference of the level D-2 values (zero outside 0..D-2)
        R a0 = (r <= D - 2) ? l2[r] : R(0);
        R a1 = (r - 1 >= 0 && r - 1 <= D - 2) ? l2[r - 1] : R(0);
        R a2 = (r - 2 >= 0 && r - 2 <= D - 2) ? l2[r - 2] : R(0);
        m[r] += h2 * (a0 - R(2) * a1 + a2);
    }
    if (D >= 4) {
        const R h4 = h * h * h * h * R(1.0 / 1920.0);
#pragma unroll
        for (int r = 0; r <= D; ++r) {
            // fourth difference of the level D-4 values
            R s = R(0);
            const R c4[5] = {R(1), R(-4), R(6), R(-4), R(1)};
#pragma unroll
            for (int q = 0; q <= 4; ++q) {
                int i = r - q;
                if (i >= 0 && i <= D - 4) s += c4[q] * l4[i];
            }
            m[r] += h4 * s;
        }
    }
}

// Walk the straight path from local offset t0 (in cell 0) by the signed
// displacement d (cell units), split at every knot (Sec. 4.2: the path integral
// of Lambda_1 along x^n -> x^{n+1}).  For each piece, visit(c, h, m) gets the
// cell c relative to the start cell, the signed piece length h (cells) and the
// means m[r] of the degree-(K-1) pieces over it.  The path integral of
// Lambda^1_{c0+c-r} over the piece is dx * h * m[r]; the path mean is the
// sum over pieces of (h/d) m[r] (or m[r] itself for a single piece).
// Returns the number of pieces.
template <int K, typename R, class Visit>
__device__ __forceinline__ int walk_path(R t0, R d, Visit &&visit)
{
    constexpr int D = K - 1;
    R m[D + 1];
    const R s = t0 + d;
    const int cend = (int)floor_(s);
    if (cend == 0) {
        piece_means<D, R>(R(0.5) * (t0 + s), d, m);
        visit(0, d, m, true);
        return 1;
    }
    int n = 0;
    if (cend > 0) {
        piece_means<D, R>(R(0.5) * (t0 + R(1)), R(1) - t0, m);
        visit(0, R(1) - t0, m, false); ++n;
        for (int c = 1; c < cend; ++c) {
            piece_means<D, R>(R(0.5), R(1), m);
            visit(c, R(1), m, false); ++n;
        }
        const R tl = s - R(cend);
        if (tl > R(0)) {
            piece_means<D, R>(R(0.5) * tl, tl, m);
            visit(cend, tl, m, false); ++n;
        }
    } else {
        if (t0 > R(0)) {
            piece_means<D, R>(R(0.5) * t0, -t0, m);
            visit(0, -t0, m, false); ++n;
        }
        for (int c = -1; c > cend; --c) {
            piece_means<D, R>(R(0.5), R(-1), m);
            visit(c, R(-1), m, false); ++n;
        }
        const R tl = s - R(cend);          // in [0,1): the piece runs from 1 down to tl
        piece_means<D, R>(R(0.5) * (R(1) + tl), tl - R(1), m);
        visit(cend, tl - R(1), m, false); ++n;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Accumulators of the per-lane deposit windows.  A lane adds the contributions of
// the markers it holds between two flushes (about a hundred at 5e4 markers a
// cell); what it adds are float values in the float form.
//  AccNative<R>: a plain R sum (the double form; the float form's fastest choice,
//                whose rounding grows with the number of markers a lane adds).
//  AccComp:      a compensated float pair (hi, lo): each add is an error-free
//                two-sum, so hi + lo carries the lane's sum to about double
//                accuracy (Knuth's TwoSum; the pair is read out in double).
//  AccDouble:    a double sum of float values (exact adds of the products,
//                on the FP64 pipe).
// warp_part() sums a slot over the warp in the accumulator's own type; value()
// converts such a sum to double (done by the one lane that writes it).
// ---------------------------------------------------------------------------
template <typename R>
struct AccNative {
    R v;
    __device__ __forceinline__ void clear() { v = R(0); }
    template <typename T> __device__ __forceinline__ void add(T x) { v += x; }
    // sum over the warp, in every lane, in the accumulator's own precision;
    // value() reads a sum out in double (called by the writing lane only)
    using Part = R;
    __device__ __forceinline__ Part warp_part() const
    {
        R t = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        return t;
    }
    __device__ __forceinline__ static double value(Part t) { return (double)t; }
};

// Knuth's TwoSum: a + b = s + e exactly (float, any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Compensated float pair with a bias: hi starts at 2^BL, far above any lane sum
// of the deposits it collects, so every add satisfies |hi| >= |x| and Dekker's
// Fast2Sum (three operations) recovers its rounding error exactly into lo, and
// hi - 2^BL is exact at read-out (Sterbenz, as long as the lane sum stays below
// 2^(BL-1)).  The sweeps take 2^BL = 4096 K! (rounded up to a power of two): their
// values are at most about K! in the scaled units of bspline_scaled, so a lane may
// collect some two thousand full-size values between flushes.  The error left is
// lo's own rounding: each add's error is at most ulp(2^BL)/2 (about 1e-3 K!), so
// lo stays a small random sum whose rounding is near 1e-11 of the lane sum, against
// about eps sqrt(n) of the sum for a plain float sum of n markers.
template <int BL>
struct AccComp {
    float hi, lo;
    static constexpr float bias() { return (float)(1u << BL); }
    __device__ __forceinline__ void clear() { hi = bias(); lo = 0.f; }
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x;
        lo += x - (s - hi);
        hi = s;
    }
    // the warp sum of (hi - bias) + lo as a float pair (the butterfly adds pairs
    // with TwoSum, so no float rounding of the partial sums is lost); value()
    // reads the pair out in double
    using Part = float2;
    __device__ __forceinline__ Part warp_part() const
    {
        float h = hi - bias(), l = lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
            float sum, e;
            two_sum(h, h2, sum, e);
            h = sum;
            l = (l + l2) + e;
        }
        return make_float2(h, l);
    }
    __device__ __forceinline__ static double value(Part t) { return (double)t.x + (double)t.y; }
};

// log2 of the bias for degree K: 12 + ceil(log2 K!)
template <int K> struct CompBias;
template <> struct CompBias<2> { static constexpr int v = 13; };
template <> struct CompBias<3> { static constexpr int v = 15; };
template <> struct CompBias<4> { static constexpr int v = 17; };
template <> struct CompBias<5> { static constexpr int v = 19; };

struct AccDouble {
    double v;
    __device__ __forceinline__ void clear() { v = 0.0; }
    __device__ __forceinline__ void add(float x) { v += (double)x; }
    __device__ __forceinline__ void add(double x) { v += x; }
    using Part = double;
    __device__ __forceinline__ Part warp_part() const
    {
        double t = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        return t;
    }
    __device__ __forceinline__ static double value(Part t) { return t; }
};

// accumulator kinds of the sweeps (pic_config.deposit), for degree K
enum : int { ACC_NATIVE = 0, ACC_COMP = 1, ACC_DOUBLE = 2 };
template <typename R, int ACC, int K> struct AccOf;
template <typename R, int K> struct AccOf<R, ACC_NATIVE, K> { using T = AccNative<R>; };
template <typename R, int K> struct AccOf<R, ACC_COMP, K> { using T = AccComp<CompBias<K>::v>; };
template <typename R, int K> struct AccOf<R, ACC_DOUBLE, K> { using T = AccDouble; };
// the accumulator a form uses unless asked otherwise
template <typename R> struct DefaultAcc { static constexpr int v = std::is_same<R, float>::value ? ACC_COMP : ACC_NATIVE; };

// ---------------------------------------------------------------------------
// Per-warp register window for deposits of cell-sorted markers.  Each lane keeps
// NS partial sums for the consecutive grid nodes b0 .. b0+NS-1 around the warp's
// base cell; a piece whose NV values fall on nodes cp - r (r = 0..NV-1) goes to
// slots (cp - base) + OFF - r, chosen by a switch so that the array stays in
// registers.  When the warp's base cell advances by one (the common case for
// sorted markers) only the lowest slot leaves the window: it is summed over the
// warp and added to the block's shared-memory row, and the other slots move
// down; any other change of base flushes every slot.  Warp sums of the plain
// float accumulator are formed in float; those of the compensated pair as float
// pairs; only the one value written per node is converted to double (GB300's
// FP64 pipe is narrow, so the window keeps double arithmetic out of its loop).
// ---------------------------------------------------------------------------
template <typename R, int NS, int NV, int OFF, int OMIN, int OMAX, typename A = AccNative<R>, bool TRACK = false>
struct DepWindow {
    A acc[NS];
    // with TRACK: this lane added to the window since its last full flush, so that
    // moves and flushes of a window nobody wrote to (e.g. A_z = 0) cost one vote
    bool dirty;
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int s = 0; s < NS; ++s) acc[s].clear();
        dirty = false;
    }
    template <int O>
    __device__ __forceinline__ void add_at(const R *v)
    {
#pragma unroll
        for (int r = 0; r < NV; ++r) acc[O + OFF - r].add(v[r]);
        dirty = true;
    }
    // returns false when the piece lies outside the window (caller takes the slow path)
    __device__ __forceinline__ bool put(int o, const R *v)
    {
        static_assert(OMIN >= -3 && OMAX <= 3 && OMIN <= 0 && OMAX >= 0, "window offsets");
        switch (o) {
        case -3: if (OMIN <= -3) { add_at<(OMIN <= -3 ? -3 : 0)>(v); return true; } return false;
        case -2: if (OMIN <= -2) { add_at<(OMIN <= -2 ? -2 : 0)>(v); return true; } return false;
        case -1: if (OMIN <= -1) { add_at<(OMIN <= -1 ? -1 : 0)>(v); return true; } return false;
        case 0: add_at<0>(v); return true;
        case 1: if (OMAX >= 1) { add_at<(OMAX >= 1 ? 1 : 0)>(v); return true; } return false;
        case 2: if (OMAX >= 2) { add_at<(OMAX >= 2 ? 2 : 0)>(v); return true; } return false;
        case 3: if (OMAX >= 3) { add_at<(OMAX >= 3 ? 3 : 0)>(v); return true; } return false;
        default: return false;
        }
    }
    // slot S summed over the warp, added (times `scale`, in double) to s_row[row0 + S]
    // by lane 0; all 32 lanes must call.  The warp sum stays in the accumulator's
    // own type and only the writing lane converts it: the double arithmetic of a
    // flush is then one lane's, not the warp's.
    template <int S>
    __device__ __forceinline__ void flush_slot(double *s_row, int row0, double scale)
    {
        const typename A::Part t = acc[S].warp_part();
        if ((threadIdx.x & 31) == 0) {
            const double v = A::value(t);
            if (v != 0.0) atomicAdd(&s_row[row0 + S], scale * v);
        }
        acc[S].clear();
    }
    // every slot to the row (row0 = shared-memory index of slot 0): lane s keeps the
    // warp sum of slot s, and lanes 0..NS-1 convert and write in one step; all
    // lanes call
    __device__ __forceinline__ void flush(double *s_row, int row0, double scale)
    {
        if (TRACK && !__any_sync(0xffffffffu, dirty)) return;     // every slot is clear
        dirty = false;
        const int lane = threadIdx.x & 31;
        typename A::Part mine{};
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const typename A::Part t = acc[q].warp_part();
            if (lane == q) mine = t;
            acc[q].clear();
        }
        if (lane < NS) {
            const double v = A::value(mine);
            if (v != 0.0) atomicAdd(&s_row[row0 + lane], scale * v);
        }
    }
    // the warp's base cell moved by `d` (warp-uniform); row0 = index of slot 0 for
    // the old base.  All lanes must call.
    __device__ __forceinline__ void advance(int d, double *s_row, int row0, double scale)
    {
        if (TRACK && !__any_sync(0xffffffffu, dirty)) return;     // nothing to move
        if (d == 1) {
            flush_slot<0>(s_row, row0, scale);
#pragma unroll
            for (int q = 0; q + 1 < NS; ++q) acc[q] = acc[q + 1];
            acc[NS - 1].clear();
        } else if (d == -1) {
            flush_slot<NS - 1>(s_row, row0, scale);
#pragma unroll
            for (int q = NS - 1; q > 0; --q) acc[q] = acc[q - 1];
            acc[0].clear();
        } else {
            flush(s_row, row0, scale);
        }
    }
};

// Cell of a marker as its warp's deposit window sees it.  Markers are sorted by
// cell, but between sorts a marker that crossed the periodic boundary carries
// cell 0, 1, .. among neighbours at cell M-1 (or the reverse): the warp's lowest
// cell is then 0, and every marker at the top end would miss the window and take
// the slow shared-atomic path.  In a warp that holds cells in the upper half of
// the grid, cells below U are shifted by +M.  Shared arrays staged with a periodic
// halo of H cells hold cell c at index c + H for -H <= c < M + H, so a kernel whose
// accesses reach at most `reach` cells above a marker's cell passes
// U = H - reach: every index stays below M + 2H.  All lanes must call.
__device__ __forceinline__ int warp_unwrap_cell(int c, bool act, int M, int U)
{
    const int hi = __reduce_max_sync(0xffffffffu, act ? c : INT_MIN);
    return (act && hi >= M / 2 && c < U) ? c + M : c;
}

// ---------------------------------------------------------------------------
// Scaled B-spline arithmetic for the sweep kernels.  A rounded reciprocal such
// as 1/3 (in float 1 + 3e-8 too large) would scale every basis value by the same
// factor; through the discrete-gradient identity such a systematic bias becomes a
// steady energy drift.  So the kernels use integer-coefficient forms and fold all
// normalisations into the double-precision staging of the fields and the
// double-precision flush of the deposits:
//   bspline_scaled<D>:  v[r] = D! N^D(r + t)  (triangle without the 1/n factors)
//   piece_means_scaled<D>: m[r] = S_D * (mean of N^D(r + t) over the piece), with
//   S_D = X_D D! chosen so that every coefficient of the midpoint formula is a
//   dyadic rational (X_1 = 1, X_2 = 3, X_3 = 1, X_4 = 5); whole-cell means are
//   then small integers, e.g. (1, 4, 1) for D = 2.
// ---------------------------------------------------------------------------
template <int D> struct MeanScale;
template <> struct MeanScale<0> { static constexpr int X = 1, S = 1; };
template <> struct MeanScale<1> { static constexpr int X = 1, S = 1; };
template <> struct MeanScale<2> { static constexpr int X = 3, S = 6; };
template <> struct MeanScale<3> { static constexpr int X = 1, S = 6; };
template <> struct MeanScale<4> { static constexpr int X = 5, S = 120; };

template <int D> struct Fact { static constexpr int v = D * Fact<D - 1>::v; };
template <> struct Fact<0> { static constexpr int v = 1; };

template <int D, typename R>
__device__ __forceinline__ void bspline_scaled(R t, R *v)
{
    v[0] = R(1);
#pragma unroll
    for (int n = 1; n <= D; ++n) {
        v[n] = (R(1) - t) * v[n - 1];
#pragma unroll
        for (int r = n - 1; r >= 1; --r) v[r] = (t + R(r)) * v[r] + (R(n + 1 - r) - t) * v[r - 1];
        v[0] = t * v[0];
    }
}

// m[r] = S_D * mean over [tm - h/2, tm + h/2] of N^D(r + t), exact for D <= 4:
// mean = f(tm) + f'' h^2/24 + f'''' h^4/1920 with f'' and f'''' from the
// second and fourth differences of the lower levels of the (scaled) triangle.
template <int D, typename R>
__device__ __forceinline__ void piece_means_scaled(R tm, R h, R *m)
{
    static_assert(D >= 1 && D <= 4, "piece degree");
    constexpr int X = MeanScale<D>::X;
    R l2[D + 1], l4[D + 1];
    m[0] = R(1);
    if (D == 2) l2[0] = R(1);
    if (D == 4) l4[0] = R(1);
#pragma unroll
    for (int n = 1; n <= D; ++n) {
        m[n] = (R(1) - tm) * m[n - 1];
#pragma unroll
        for (int r = n - 1; r >= 1; --r) m[r] = (tm + R(r)) * m[r] + (R(n + 1 - r) - tm) * m[r - 1];
        m[0] = tm * m[0];
        if (n == D - 2) {
#pragma unroll
            for (int r = 0; r <= (D - 2 > 0 ? D - 2 : 0); ++r) l2[r] = m[r];
        }
        if (n == D - 4) {
#pragma unroll
            for (int r = 0; r <= (D - 4 > 0 ? D - 4 : 0); ++r) l4[r] = m[r];
        }
    }
    if (D >= 2) {
        // X D! N'' h^2/24 = h^2 * (X D (D-1) / 24) * (second difference of (D-2)! N^{D-2})
        const R c2 = R(X * D * (D - 1)) / R(24);           // 1/4, 1/4, 5/2: dyadic
        const R hh = h * h * c2;
#pragma unroll
        for (int r = 0; r <= D; ++r) {
            R a0 = (r <= D - 2) ? l2[r] : R(0);
            R a1 = (r - 1 >= 0 && r - 1 <= D - 2) ? l2[r - 1] : R(0);
            R a2 = (r - 2 >= 0 && r - 2 <= D - 2) ? l2[r - 2] : R(0);
            m[r] = R(X) * m[r] + hh * (a0 - R(2) * a1 + a2);
        }
    } else {
#pragma unroll
        for (int r = 0; r <= D; ++r) m[r] = R(X) * m[r];
    }
    if (D >= 4) {
        // X D! N'''' h^4/1920 = h^4 * (X D(D-1)(D-2)(D-3) / 1920) * (fourth difference of N^0)
        const R c4 = R(X * D * (D - 1) * (D - 2) * (D - 3)) / R(1920);   // 1/16
        const R h4 = h * h * h * h * c4;
        const R d4[5] = {R(1), R(-4), R(6), R(-4), R(1)};
#pragma unroll
        for (int r = 0; r <= D; ++r) {
            R s = R(0);
#pragma unroll
            for (int q = 0; q <= 4; ++q) {
                const int i = r - q;
                if (i >= 0 && i <= D - 4) s += d4[q] * l4[i];
            }
            m[r] += h4 * s;
        }
    }
}

// Number of pieces of the path from local offset t0 by d cells: 1 + knots crossed.
template <typename R>
__device__ __forceinline__ int path_pieces(R t0, R d)
{
    return abs((int)floor_(t0 + d)) + 1;
}

template <typename R> __device__ __forceinline__ R clamp01(R v) { return v < R(0) ? R(0) : (v > R(1) ? R(1) : v); }

// Branch-free walk of the path t0 -> s = t0 + d split at knots.  Piece p lies in
// cell c = sign(d) p relative to the start cell.  The piece lengths are formed
// from d and the knot distances, never as differences of clamped coordinates,
// so a single-piece path has length exactly d:
//   one piece:   t0 -> s                       (h = d)
//   first piece: t0 -> the knot ahead           (h = 1 - t0, or -t0 moving left)
//   middle:      a whole cell                   (h = +-1, midpoint 1/2)
//   last piece:  the knot behind -> tl = s - floor(s)  (h = tl, or tl - 1 moving left)
// The caller passes the warp maximum of the piece counts, so every lane runs the
// same trip count; pieces beyond a lane's own count have zero length.
// visit(c, h, m, p) gets the signed piece length h (cells) and the scaled means
// m[r] = S_{K-1} * mean of the degree-(K-1) pieces over it (piece_means_scaled).
template <int K, typename R, class Visit>
__device__ __forceinline__ void walk_uniform(R t0, R d, int npc, Visit &&visit)
{
    constexpr int D = K - 1;
    const R s = t0 + d;
    const R fl = floor_(s);
    const int n = abs((int)fl) + 1;          // this lane's piece count
    const R tl = s - fl;                     // local offset of the end point
    const bool right = d >= R(0);
    const int sg = right ? 1 : -1;
    R m[D + 1];
    for (int p = 0; p < npc; ++p) {
        R h, tm;
        if (n == 1) {
            h = (p == 0) ? d : R(0);
            tm = R(0.5) * (t0 + s);
        } else if (p == 0) {
            h = right ? R(1) - t0 : -t0;
            tm = t0 + R(0.5) * h;
        } else if (p == n - 1) {
            h = right ? tl : tl - R(1);
            tm = R(0.5) * (right ? tl : R(1) + tl);
        } else if (p < n) {
            h = R(sg);
            tm = R(0.5);
        } else {
            h = R(0);
            tm = R(0.5);
        }
        piece_means_scaled<D, R>(tm, h, m);
        visit(sg * p, h, m, p);
    }
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v || w != w) ? w : v;       // NaN wins
    }
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide max of a non-negative double, then one atomicMax per block.
__device__ __forceinline__ void block_max_to(unsigned long long *dst, double v, double *s_red)
{
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double u = lane < nw ? s_red[lane] : 0.0;
        u = warp_max(u);
        if (lane == 0) atomic_max_nonneg(dst, u);
    }
    __syncthreads();
}

__device__ __forceinline__ void block_sum_to(double *dst, double v, double *s_red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double u = lane < nw ? s_red[lane] : 0.0;
        u = warp_sum(u);
        if (lane == 0) atomicAdd(dst, u);
    }
    __syncthreads();
}

}  // namespace pic
