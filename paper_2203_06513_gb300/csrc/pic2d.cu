// pic2d.cu -- subsystem I of the two-dimensional scheme (Sec. 4.3) on the GPU, FP64.
//
// Spaces (Sec. 3.2): tensor-product B-splines on a uniform periodic M1 x M2 grid,
// node i = i1 * M2 + i2; A_z on N^k x N^k, the 1-form e_xy as e_x on N^{k-1} x N^k
// and e_y on N^k x N^{k-1}.  One thread per marker and sweep:
//   * the path means of both V1 components along x^n -> x^(k) (the straight path
//     split at every knot crossing of either coordinate, k-point Gauss--Legendre on
//     each piece: the integrand is a polynomial of degree 2k - 1 there), gathered
//     against e_bar;
//   * the coordinate-increment difference quotients D of A_z as exact path means of
//     dA/dx1 along x1 (at x2^(k)) and of dA/dx2 along x2 (at x1^n);
//   * with spins (hbar != 0), the quotients of the Zeeman term hbar s . B,
//     B = (dA/dx2, -dA/dx1, b_z), the same way: path means of the second
//     differences of A_z and the first differences of b_z along each coordinate;
//   * the momentum and position updates of the discrete-gradient scheme;
//   * the current of the new path x^n -> x^(k+1), accumulated per block in shared
//     memory over the whole grid and added to the global deposit once per node.
// The grid side applies M1^{-1} = diag(M1_x^{-1} (x) M0_y^{-1}, M0_x^{-1} (x) M1_y^{-1})
// as two circulant passes with the exact inverse rows of the 1D mass matrices.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pic2d.h"
#include "pic_internal.h"

namespace pic {
namespace {

constexpr int kMax2DNodes = 4096;     // M1 * M2: the block's shared-memory deposit rows
constexpr int kMaxCross = 16;         // knot crossings per coordinate and path

struct Args2D {
    int M1, M2;
    long long np;
    double dx1, dx2, dt, w;
    double idx1, idx2;      // 1 / dx1, 1 / dx2
    const double *x;        // np x 2, in the box
    double *a0;             // np: A_z(x^n), written by the first sweep of a step
    int first;              // this is the step's first sweep
    const double *pn;       // np x 2
    double *d;              // np x 2 displacement iterate (length units), in/out
    double *pk;             // np x 2 momentum iterate, in/out
    const double *ebx, *eby;
    const double *az, *gax, *gay;
    double *jx, *jy;        // deposits of this sweep (zeroed before)
    double hbar;            // Zeeman terms on when non-zero (spins given)
    const double *s;        // np x 3 spins
    const double *gxy, *gxx, *gyy, *gbx, *gby;   // G_x G_y a, G_x G_x a, G_y G_y a, G_x b_z, G_y b_z
    unsigned long long *dmax_bits, *pmax_bits;
    int *status;
    double glx[5], glw[5];  // K-point Gauss--Legendre on [-1, 1]
};

__device__ __forceinline__ int wrapi(int i, int M)
{
    int r = i % M;
    return r < 0 ? r + M : r;
}

// [N^D(r + t)], r = 0..D: the normalised B-spline values of one cell
template <int D>
__device__ __forceinline__ void bsp(double t, double *v)
{
    bspline_scaled<D, double>(t, v);
    const double s = 1.0 / (double)Fact<D>::v;
#pragma unroll
    for (int r = 0; r <= D; ++r) v[r] *= s;
}

// Pieces of the path u0 -> u0 + du (cell units, both coordinates) between knot
// crossings: f(sa, sb) for consecutive parameter values 0 = s_0 < ... = 1.
// Returns false when a coordinate crosses more than kMaxCross knots.
template <class F>
__device__ __forceinline__ bool walk2(double u0x, double u0y, double dux, double duy, F &&f)
{
    const double ex = u0x + dux, ey = u0y + duy;
    const int tx = dux > 0.0 ? (int)ceil(ex) - 1 - (int)floor(u0x) : (dux < 0.0 ? (int)ceil(u0x) - 1 - (int)floor(ex) : 0);
    const int ty = duy > 0.0 ? (int)ceil(ey) - 1 - (int)floor(u0y) : (duy < 0.0 ? (int)ceil(u0y) - 1 - (int)floor(ey) : 0);
    if (tx > kMaxCross || ty > kMaxCross) return false;
    // next knot index and its step in each coordinate; crossing parameters by the
    // reciprocal of the increment
    int nx = dux > 0.0 ? (int)floor(u0x) + 1 : (int)ceil(u0x) - 1;
    int ny = duy > 0.0 ? (int)floor(u0y) + 1 : (int)ceil(u0y) - 1;
    const int sx = dux > 0.0 ? 1 : -1, sy = duy > 0.0 ? 1 : -1;
    const double rx = tx > 0 ? 1.0 / dux : 0.0, ry = ty > 0 ? 1.0 / duy : 0.0;
    int cx = 0, cy = 0;
    double sa = 0.0;
    for (int guard = 0; guard < 2 * kMaxCross + 2; ++guard) {
        const double bx = cx < tx ? ((double)nx - u0x) * rx : 2.0;
        const double by = cy < ty ? ((double)ny - u0y) * ry : 2.0;
        const double sb = fmin(fmin(bx, by), 1.0);
        if (sb > sa) f(sa, sb);
        if (sb >= 1.0) return true;
        if (bx <= sb) { nx += sx; ++cx; }
        if (by <= sb) { ny += sy; ++cy; }
        sa = sb;
    }
    return true;
}

// 1D pieces of u0 -> u0 + du
template <class F>
__device__ __forceinline__ bool walk1(double u0, double du, F &&f)
{
    return walk2(u0, 0.0, du, 0.0, [&](double sa, double sb) { f(sa, sb); });
}

// One triangle for two degrees: vk[r] = D! N^D(r + t) (r = 0..D) and
// vm[r] = (D-1)! N^{D-1}(r + t) (r = 0..D-1), both left unnormalised
template <int D>
__device__ __forceinline__ void bsp_pair(double t, double *vk, double *vm)
{
    vk[0] = 1.0;
    if (D == 1) vm[0] = 1.0;
#pragma unroll
    for (int n = 1; n <= D; ++n) {
        vk[n] = (1.0 - t) * vk[n - 1];
#pragma unroll
        for (int r = n - 1; r >= 1; --r) vk[r] = (t + (double)r) * vk[r] + ((double)(n + 1 - r) - t) * vk[r - 1];
        vk[0] = t * vk[0];
        if (n == D - 1) {
#pragma unroll
            for (int r = 0; r < D; ++r) vm[r] = vk[r];
        }
    }
}

// sum_i c_i N^{D1}(u1 - i1) N^{D2}(u2 - i2) at one point (cell coordinates)
template <int D1, int D2>
__device__ __forceinline__ double value_dd(const double *c, int M1, int M2, double u1, double u2)
{
    const double c1 = floor(u1), c2 = floor(u2);
    double v1[D1 + 1], v2[D2 + 1];
    bspline_scaled<D1, double>(u1 - c1, v1);
    bspline_scaled<D2, double>(u2 - c2, v2);
    int o2[D2 + 1];
#pragma unroll
    for (int r2 = 0; r2 <= D2; ++r2) o2[r2] = wrapi((int)c2 - r2, M2);
    double s = 0.0;
#pragma unroll
    for (int r1 = 0; r1 <= D1; ++r1) {
        const double *row = c + wrapi((int)c1 - r1, M1) * M2;
        double t = 0.0;
#pragma unroll
        for (int r2 = 0; r2 <= D2; ++r2) t = fma(v2[r2], row[o2[r2]], t);
        s = fma(v1[r1], t, s);
    }
    return s * (1.0 / ((double)Fact<D1>::v * (double)Fact<D2>::v));
}

template <int K>
__device__ __forceinline__ double value0(const double *a, int M1, int M2, double u1, double u2)
{
    return value_dd<K, K>(a, M1, M2, u1, u2);
}

// The basis weights of one knot piece [sa, sb] of the path u0 -> u0 + du (inside
// the cell (c1, c2)): mx[r1][r2] = (sb - sa) x the mean over the piece of the
// x-component basis N^{K-1} x N^K at node (c1 - r1, c2 - r2), my likewise for the
// y-component N^K x N^{K-1}, both times (K-1)! K! (unnormalised B-splines).
// K-point Gauss--Legendre is exact: the integrand is a polynomial of degree
// 2K - 1 in the path parameter.
template <int K>
__device__ __forceinline__ void piece_weights(const Args2D &A, double u0x, double u0y, double dux, double duy,
                                              double sa, double sb, double c1, double c2, double (&mx)[K][K + 1],
                                              double (&my)[K + 1][K])
{
    const double sm = 0.5 * (sa + sb), hs = 0.5 * (sb - sa);
#pragma unroll
    for (int g = 0; g < K; ++g) {
        const double s = fma(hs, A.glx[g], sm);
        const double wq = hs * A.glw[g];
        double b1k[K + 1], b1m[K], b2k[K + 1], b2m[K];
        bsp_pair<K>(fma(s, dux, u0x) - c1, b1k, b1m);
        bsp_pair<K>(fma(s, duy, u0y) - c2, b2k, b2m);
#pragma unroll
        for (int r1 = 0; r1 < K; ++r1) {
            const double f = wq * b1m[r1];
#pragma unroll
            for (int r2 = 0; r2 <= K; ++r2) mx[r1][r2] = g == 0 ? f * b2k[r2] : fma(f, b2k[r2], mx[r1][r2]);
        }
#pragma unroll
        for (int r1 = 0; r1 <= K; ++r1) {
            const double f = wq * b1k[r1];
#pragma unroll
            for (int r2 = 0; r2 < K; ++r2) my[r1][r2] = g == 0 ? f * b2m[r2] : fma(f, b2m[r2], my[r1][r2]);
        }
    }
}

// node offsets of the cell (c1, c2): o1[r] = ((c1 - r) mod M1) M2, o2[r] = (c2 - r) mod M2
template <int K>
__device__ __forceinline__ void cell_offsets(const Args2D &A, double c1, double c2, int *o1, int *o2)
{
#pragma unroll
    for (int r = 0; r <= K; ++r) {
        o1[r] = wrapi((int)c1 - r, A.M1) * A.M2;
        o2[r] = wrapi((int)c2 - r, A.M2);
    }
}

// (Ex, Ey) = the path means of e_bar's two components along u0 -> u0 + du
template <int K>
__device__ __forceinline__ bool gather_path(const Args2D &A, double u0x, double u0y, double dux, double duy,
                                            double &Ex, double &Ey)
{
    double sx = 0.0, sy = 0.0;
    const bool ok = walk2(u0x, u0y, dux, duy, [&](double sa, double sb) {
        const double sm = 0.5 * (sa + sb);
        const double c1 = floor(fma(sm, dux, u0x)), c2 = floor(fma(sm, duy, u0y));
        double mx[K][K + 1], my[K + 1][K];
        piece_weights<K>(A, u0x, u0y, dux, duy, sa, sb, c1, c2, mx, my);
        int o1[K + 1], o2[K + 1];
        cell_offsets<K>(A, c1, c2, o1, o2);
#pragma unroll
        for (int r1 = 0; r1 <= K; ++r1) {
            const double *rx = A.ebx + o1[r1], *ry = A.eby + o1[r1];
#pragma unroll
            for (int r2 = 0; r2 <= K; ++r2) {
                if (r1 < K) sx = fma(mx[r1 < K ? r1 : 0][r2], rx[o2[r2]], sx);
                if (r2 < K) sy = fma(my[r1][r2 < K ? r2 : 0], ry[o2[r2]], sy);
            }
        }
    });
    const double scale = 1.0 / ((double)Fact<K - 1>::v * (double)Fact<K>::v);
    Ex = sx * scale;
    Ey = sy * scale;
    return ok;
}

// s_j[x | y] += (wx, wy) x the path means of the two basis components along
// u0 -> u0 + du, one shared-memory add per node and knot piece
template <int K>
__device__ __forceinline__ bool deposit_path(const Args2D &A, double *s_j, int N, double u0x, double u0y, double dux,
                                             double duy, double wx, double wy)
{
    const double scale = 1.0 / ((double)Fact<K - 1>::v * (double)Fact<K>::v);
    const double cx = wx * scale, cy = wy * scale;
    return walk2(u0x, u0y, dux, duy, [&](double sa, double sb) {
        const double sm = 0.5 * (sa + sb);
        const double c1 = floor(fma(sm, dux, u0x)), c2 = floor(fma(sm, duy, u0y));
        double mx[K][K + 1], my[K + 1][K];
        piece_weights<K>(A, u0x, u0y, dux, duy, sa, sb, c1, c2, mx, my);
        int o1[K + 1], o2[K + 1];
        cell_offsets<K>(A, c1, c2, o1, o2);
#pragma unroll
        for (int r1 = 0; r1 <= K; ++r1) {
#pragma unroll
            for (int r2 = 0; r2 <= K; ++r2) {
                const int i = o1[r1] + o2[r2];
                if (r1 < K && cx != 0.0) atomicAdd(&s_j[i], cx * mx[r1 < K ? r1 : 0][r2]);
                if (r2 < K && cy != 0.0) atomicAdd(&s_j[N + i], cy * my[r1][r2 < K ? r2 : 0]);
            }
        }
    });
}

// mean of dA/dx1 along x1 from u0 to u0 + du at fixed x2 (cell coordinate uo):
// sum (G_x a)_i (mean of N^{K-1}(x1 - i1)) N^K(x2 - i2); and the same along x2.
// The across factor is contracted once per knot piece; the along factor is the
// exact piece mean of the midpoint form (no quadrature nodes).
template <int K>
__device__ __forceinline__ double dA_mean(const Args2D &A, int axis, double u0, double du, double uo)
{
    const double co = floor(uo);
    double vo[K + 1];
    bspline_scaled<K, double>(uo - co, vo);
    const double *ga = axis == 0 ? A.gax : A.gay;
    const int Ma = axis == 0 ? A.M1 : A.M2, Mo = axis == 0 ? A.M2 : A.M1;
    const int sa_ = axis == 0 ? A.M2 : 1, so = axis == 0 ? 1 : A.M2;
    int io[K + 1];
#pragma unroll
    for (int ro = 0; ro <= K; ++ro) io[ro] = wrapi((int)co - ro, Mo) * so;
    double s = 0.0;
    walk1(u0, du, [&](double pa, double pb) {
        const double sm = 0.5 * (pa + pb), hs = 0.5 * (pb - pa);
        const double c = floor(fma(sm, du, u0));
        double col[K];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const double *q = ga + wrapi((int)c - r, Ma) * sa_;
            double acc = 0.0;
#pragma unroll
            for (int ro = 0; ro <= K; ++ro) acc = fma(q[io[ro]], vo[ro], acc);
            col[r] = acc;
        }
        // the exact mean of the degree-(K-1) pieces over this piece (midpoint form,
        // S_{K-1} times the mean), times its parameter length and (K-1)! / S_{K-1}
        double m[K];
        piece_means_scaled<K - 1, double>(fma(sm, du, u0) - c, 2.0 * hs * du, m);
        double v = 0.0;
#pragma unroll
        for (int r = 0; r < K; ++r) v = fma(m[r], col[r], v);
        constexpr double kPM = (double)Fact<K - 1>::v / (double)MeanScale<K - 1>::S;
        s = fma(2.0 * hs * kPM, v, s);
    });
    return s * (1.0 / ((double)Fact<K - 1>::v * (double)Fact<K>::v));
}

// One coordinate-increment quotient of the Zeeman term along `axis`: the mean over
// u_axis in [u0, u0 + du] (the other coordinate fixed at uo) of
//   wm dF_m/du + wp dF_p/du + wb dF_b/du,
// given the derivative coefficients on their own degrees (along, across):
// cm on (K-1, K-1), cp on (K-2, K), cb on (K-2, K-1).  Along x1 these are
// G_x G_y a, G_x G_x a and G_x b_z; along x2, G_x G_y a, G_y G_y a and G_y b_z.
template <int K>
__device__ __forceinline__ double zee_mean(const Args2D &A, int axis, double u0, double du, double uo,
                                           const double *cm, double wm, const double *cp, double wp,
                                           const double *cb, double wb)
{
    const double co = floor(uo);
    double vk[K + 1], vm[K];
    bsp_pair<K>(uo - co, vk, vm);
    // normalisations of the unnormalised values folded into the weights
    constexpr double fk = (double)Fact<K>::v, fm = (double)Fact<K - 1>::v, f2 = (double)Fact<K - 2>::v;
    const double em = wm * (1.0 / (fm * fm)), ep = wp * (1.0 / (f2 * fk)), eb = wb * (1.0 / (f2 * fm));
    const int Ma = axis == 0 ? A.M1 : A.M2, Mo = axis == 0 ? A.M2 : A.M1;
    const int sa = axis == 0 ? A.M2 : 1, so = axis == 0 ? 1 : A.M2;
    int io[K + 1];
#pragma unroll
    for (int ro = 0; ro <= K; ++ro) io[ro] = wrapi((int)co - ro, Mo) * so;
    double s = 0.0;
    walk1(u0, du, [&](double pa, double pb) {
        const double sm = 0.5 * (pa + pb), hs = 0.5 * (pb - pa);
        const double c = floor(fma(sm, du, u0));
        double colm[K], colq[K - 1];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int ia = wrapi((int)c - r, Ma) * sa;
            double am = 0.0;
#pragma unroll
            for (int ro = 0; ro < K; ++ro) am = fma(cm[ia + io[ro]], vm[ro], am);
            colm[r] = em * am;
            if (r < K - 1) {
                double ap = 0.0, ab = 0.0;
#pragma unroll
                for (int ro = 0; ro <= K; ++ro) ap = fma(cp[ia + io[ro]], vk[ro], ap);
#pragma unroll
                for (int ro = 0; ro < K; ++ro) ab = fma(cb[ia + io[ro]], vm[ro], ab);
                colq[r < K - 1 ? r : 0] = ep * ap + eb * ab;
            }
        }
        // exact means of the degree-(K-1) and degree-(K-2) pieces over this piece
        // (midpoint form, S_D times the mean; degree 0 is 1 inside one cell), each
        // times D! / S_D to match the unnormalised values the weights expect
        const double tm = fma(sm, du, u0) - c, hh = 2.0 * hs * du;
        double m1[K], m2[K - 1];
        piece_means_scaled<K - 1, double>(tm, hh, m1);
        if constexpr (K >= 3) piece_means_scaled<(K >= 3 ? K - 2 : 1), double>(tm, hh, m2);
        else m2[0] = 1.0;
        constexpr double c1 = (double)Fact<K - 1>::v / (double)MeanScale<K - 1>::S;
        constexpr double c2 = (double)Fact<K - 2>::v / (double)MeanScale<K - 2>::S;
        double v1 = 0.0, v2 = 0.0;
#pragma unroll
        for (int r = 0; r < K; ++r) v1 = fma(m1[r], colm[r], v1);
#pragma unroll
        for (int r = 0; r < K - 1; ++r) v2 = fma(m2[r], colq[r], v2);
        s = fma(2.0 * hs, c1 * v1 + c2 * v2, s);
    });
    return s;
}

__device__ __forceinline__ void max_bits(unsigned long long *dst, double v)
{
    // non-negative doubles order like their bit patterns; NaN maps to the largest
    const unsigned long long b = (v == v) ? (unsigned long long)__double_as_longlong(v) : 0x7ff8000000000000ull;
    atomicMax(dst, b);
}

// PRE: the predicted start instead of a sweep -- A(x^n) stored, the explicit
// predictor delta^(0) = dt p^n / gamma(p^n, A(x^n)) written and the current of
// x^n -> x^n + delta^(0) deposited, so that the fixed point can start from the
// field consistent with it; no gather, no momentum update, no increments.
template <int K, bool PRE = false>
__global__ void __launch_bounds__(256, K <= 3 ? 2 : 1) k2_sweep(Args2D A)
{
    extern __shared__ double s_j[];     // 2 * M1 * M2: x then y
    __shared__ int s_perm[256];
    __shared__ int s_cnt[8];
    const int N = A.M1 * A.M2;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s_j[i] = 0.0;
    __syncthreads();
    double dm = 0.0, pm = 0.0;
    bool bad = false;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (long long base = blockIdx.x * 256LL; base < A.np; base += gridDim.x * 256LL) {
        // The block's 256 markers in two groups, paths within one cell first and
        // paths across a knot last (by the current iterate; the new path mostly
        // follows it): a warp then runs the extra pieces of a crossing only when
        // it holds crossing markers, instead of nearly every warp running them
        // for one lane.
        {
            const long long b = base + threadIdx.x;
            bool multi = true;
            if (b < A.np) {
                // the predicted start's path is within dt p (gamma >= 1)
                const double vx = A.x[2 * b] * A.idx1, vy = A.x[2 * b + 1] * A.idx2;
                const double ex = PRE ? A.dt * A.pn[2 * b] : A.d[2 * b];
                const double ey = PRE ? A.dt * A.pn[2 * b + 1] : A.d[2 * b + 1];
                multi = floor(vx + ex * A.idx1) != floor(vx) || floor(vy + ey * A.idx2) != floor(vy);
            }
            const unsigned one = __ballot_sync(0xffffffffu, !multi);
            if (lane == 0) s_cnt[wid] = __popc(one);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const int c = s_cnt[w];
                before += w < wid ? c : 0;
                total += c;
            }
            s_perm[multi ? total + (wid * 32 - before) + __popc(~one & lt) : before + __popc(one & lt)] = threadIdx.x;
            __syncthreads();
        }
        const long long a = base + s_perm[threadIdx.x];
        __syncthreads();                    // s_perm and s_cnt are free for the next group
        if (a >= A.np) continue;
        {
        const double u0x = A.x[2 * a] * A.idx1, u0y = A.x[2 * a + 1] * A.idx2;
        const double d0 = A.d[2 * a], d1 = A.d[2 * a + 1];
        const double p0 = A.pn[2 * a], p1 = A.pn[2 * a + 1];
        const double dux = d0 * A.idx1, duy = d1 * A.idx2;
        if constexpr (PRE) {
            const double A0 = value0<K>(A.az, A.M1, A.M2, u0x, u0y);
            A.a0[a] = A0;
            const double r = A.dt / sqrt(1.0 + p0 * p0 + p1 * p1 + A0 * A0);
            const double n0 = r * p0, n1 = r * p1;
            if (!deposit_path<K>(A, s_j, N, u0x, u0y, n0 * A.idx1, n1 * A.idx2, A.w * n0, A.w * n1)) bad = true;
            A.d[2 * a] = n0;
            A.d[2 * a + 1] = n1;
            continue;
        }
        // A(x^n) is the same in every sweep of the step: evaluated in the first
        double A0;
        if (A.first) {
            A0 = value0<K>(A.az, A.M1, A.M2, u0x, u0y);
            A.a0[a] = A0;
        } else {
            A0 = A.a0[a];
        }
        const double A1 = value0<K>(A.az, A.M1, A.M2, u0x + dux, u0y + duy);
        double Ex, Ey;
        bool ok = gather_path<K>(A, u0x, u0y, dux, duy, Ex, Ey);
        const double D1 = dA_mean<K>(A, 0, u0x, dux, u0y + duy);
        const double D2 = dA_mean<K>(A, 1, u0y, duy, u0x);
        const double pp = p0 * p0 + p1 * p1;
        const double g0 = sqrt(1.0 + pp + A0 * A0);
        const double g1 = sqrt(1.0 + pp + A1 * A1);
        const double f = A.dt * (A1 + A0) / (g1 + g0);
        double q0 = p0 + A.dt * Ex - f * D1;
        double q1 = p1 + A.dt * Ey - f * D2;
        if (A.hbar != 0.0) {
            // discrete gradient of hbar s . B, B = (dA/dx2, -dA/dx1, b_z)
            const double sx = A.s[3 * a], sy = A.s[3 * a + 1], sz = A.s[3 * a + 2];
            const double Z1 = zee_mean<K>(A, 0, u0x, dux, u0y + duy, A.gxy, sx, A.gxx, -sy, A.gbx, sz);
            const double Z2 = zee_mean<K>(A, 1, u0y, duy, u0x, A.gxy, -sy, A.gyy, sx, A.gby, sz);
            q0 -= A.dt * A.hbar * Z1;
            q1 -= A.dt * A.hbar * Z2;
        }
        const double g2 = sqrt(1.0 + q0 * q0 + q1 * q1 + A1 * A1);
        const double r = A.dt / (g1 + g2);
        const double n0 = r * (p0 + q0);
        const double n1 = r * (p1 + q1);
        if (!(isfinite(n0) && isfinite(n1))) { bad = true; continue; }
        // the current of the new path
        ok = ok && deposit_path<K>(A, s_j, N, u0x, u0y, n0 * A.idx1, n1 * A.idx2, A.w * n0, A.w * n1);
        if (!ok) bad = true;
        dm = fmax(dm, fmax(fabs(n0 - d0), fabs(n1 - d1)));
        pm = fmax(pm, fmax(fabs(q0 - A.pk[2 * a]), fabs(q1 - A.pk[2 * a + 1])));
        A.d[2 * a] = n0;
        A.d[2 * a + 1] = n1;
        A.pk[2 * a] = q0;
        A.pk[2 * a + 1] = q1;
        }
    }
    if (bad) atomicOr(A.status, STATUS_NUMERIC);
    // block maxima of the increments
    __shared__ double s_m[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_m[0][threadIdx.x >> 5] = dm;
        s_m[1][threadIdx.x >> 5] = pm;
    }
    __syncthreads();
    if (threadIdx.x == 0 && !PRE) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fmax(a, s_m[0][w]);
            b = fmax(b, s_m[1][w]);
        }
        max_bits(A.dmax_bits, a);
        max_bits(A.pmax_bits, b);
    }
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
        const double v = s_j[i];
        if (v != 0.0) atomicAdd(i < N ? &A.jx[i] : &A.jy[i - N], v);
    }
}

// out[i1, i2] = sum_q g[(i_axis - q) mod M_axis] in[.. q ..] along one axis
__global__ void k2_circ(int M1, int M2, int axis, const double *g, const double *in, double *out)
{
    const int N = M1 * M2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int i1 = i / M2, i2 = i % M2;
        double s = 0.0;
        if (axis == 0) {
            for (int q = 0; q < M1; ++q) s += g[wrapi(i1 - q, M1)] * in[q * M2 + i2];
        } else {
            for (int q = 0; q < M2; ++q) s += g[wrapi(i2 - q, M2)] * in[i1 * M2 + q];
        }
        out[i] = s;
    }
}

// e^(k+1) = e^n - sol (sol = M1^{-1} j); increment max-norm; e_bar for the next sweep
__global__ void k2_update(int N, const double *en, const double *sol, double *ek, double *eb,
                          unsigned long long *emax_bits)
{
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double v = en[i] - sol[i];
        m = fmax(m, fabs(v - ek[i]));
        if (!(v == v)) m = v;
        ek[i] = v;
        eb[i] = 0.5 * (en[i] + v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, m, o);
        m = (t > m || t != t) ? t : m;
    }
    if ((threadIdx.x & 31) == 0) max_bits(emax_bits, m);
}

// acc[0] += sum_a w (g(p_a, A(x_a)) - 1); with spins, acc[1] += sum_a w hbar
// (s_x dA/dx2 - s_y dA/dx1 + s_z b_z)(x_a) (G_y a on (K, K-1), G_x a on (K-1, K),
// b_z on (K-1, K-1))
template <int K>
__global__ void __launch_bounds__(256) k2_energy(long long np, int M1, int M2, double dx1, double dx2, double w,
                                                  const double *x, const double *p, const double *az, double hbar,
                                                  const double *sp, const double *gax, const double *gay,
                                                  const double *bz, double *acc)
{
    double s = 0.0, z = 0.0;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < np;
         a += (long long)gridDim.x * blockDim.x) {
        const double u1 = x[2 * a] / dx1, u2 = x[2 * a + 1] / dx2;
        const double A = value0<K>(az, M1, M2, u1, u2);
        s += w * (sqrt(1.0 + p[2 * a] * p[2 * a] + p[2 * a + 1] * p[2 * a + 1] + A * A) - 1.0);
        if (hbar != 0.0)
            z += w * hbar * (sp[3 * a] * value_dd<K, K - 1>(gay, M1, M2, u1, u2) -
                             sp[3 * a + 1] * value_dd<K - 1, K>(gax, M1, M2, u1, u2) +
                             sp[3 * a + 2] * value_dd<K - 1, K - 1>(bz, M1, M2, u1, u2));
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, s);
        if (hbar != 0.0) atomicAdd(acc + 1, z);
    }
}

// x^{n+1} = x^n + delta wrapped into the box, p^{n+1} = p^(k)
__global__ void k2_finalize(long long np, double L1, double L2, double *x, double *p, const double *d,
                            const double *pk)
{
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < np;
         a += (long long)gridDim.x * blockDim.x) {
        for (int q = 0; q < 2; ++q) {
            const double L = q == 0 ? L1 : L2;
            double v = x[2 * a + q] + d[2 * a + q];
            v -= L * floor(v / L);
            if (v >= L) v -= L;
            if (v < 0.0) v = 0.0;
            x[2 * a + q] = v;
            p[2 * a + q] = pk[2 * a + q];
        }
    }
}

// K-point Gauss--Legendre nodes and weights on [-1, 1] by Newton's method on the
// three-term recurrence of the Legendre polynomials
void gauss_legendre(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 1; j < n; ++j) {
                const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 0 ? 1.0 : p1, pm = n == 0 ? 0.0 : p0;
            if (n == 1) { pn = z; pm = 1.0; }
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace
}  // namespace pic

using namespace pic;

struct pic2d_handle {
    pic2d_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    double dx1 = 0.0, dx2 = 0.0;
    int N = 0;
    double *x = nullptr, *p = nullptr, *d = nullptr, *pk = nullptr, *a0 = nullptr;
    double *ex = nullptr, *ey = nullptr, *exk = nullptr, *eyk = nullptr, *ebx = nullptr, *eby = nullptr;
    double *az = nullptr, *gax = nullptr, *gay = nullptr;
    double *gxy = nullptr, *gxx = nullptr, *gyy = nullptr;       // second differences of a_z
    double *spin = nullptr, *bz = nullptr, *gbx = nullptr, *gby = nullptr;   // pic2d_set_spin
    double *jx = nullptr, *jy = nullptr, *tmp = nullptr, *sol = nullptr;
    double *g1x = nullptr, *g0y = nullptr, *g0x = nullptr, *g1y = nullptr;   // inverse rows
    unsigned long long *bits = nullptr;      // dmax, pmax, emax
    int *status = nullptr;
    double *acc = nullptr;
    std::vector<double> m0x, m1x, m0y, m1y;  // 1D mass rows (host) for the field energy
    double glx[5] = {0, 0, 0, 0, 0}, glw[5] = {0, 0, 0, 0, 0};
    std::string err;
};

static thread_local std::string g_err2d;

static int fail2d(pic2d_handle *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_err2d = buf;
    return code;
}

#define CK2(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail2d(h, PIC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void free2d(pic2d_handle *h)
{
    double **arrs[] = {&h->x, &h->p, &h->d, &h->pk, &h->a0, &h->ex, &h->ey, &h->exk, &h->eyk, &h->ebx, &h->eby,
                       &h->az, &h->gax, &h->gay, &h->jx, &h->jy, &h->tmp, &h->sol, &h->g1x, &h->g0y,
                       &h->g0x, &h->g1y, &h->acc,
                       &h->gxy, &h->gxx, &h->gyy, &h->spin, &h->bz, &h->gbx, &h->gby};
    for (double **a : arrs)
        if (*a) { cudaFree(*a); *a = nullptr; }
    if (h->bits) cudaFree(h->bits);
    if (h->status) cudaFree(h->status);
    h->bits = nullptr;
    h->status = nullptr;
}

// backward difference of a grid array along one axis, divided by the cell size
static std::vector<double> grid_diff(const std::vector<double> &c, int M1, int M2, int axis, double dx)
{
    std::vector<double> out(c.size());
    for (int i1 = 0; i1 < M1; ++i1)
        for (int i2 = 0; i2 < M2; ++i2) {
            const int i = i1 * M2 + i2;
            const int j = axis == 0 ? ((i1 - 1 + M1) % M1) * M2 + i2 : i1 * M2 + (i2 - 1 + M2) % M2;
            out[i] = (c[i] - c[j]) / dx;
        }
    return out;
}

// full periodic circulant row of the degree-d mass matrix (band folded onto M nodes)
static std::vector<double> mass_row_full(int d, int M, double dx)
{
    std::vector<double> band(d + 1), row(M, 0.0);
    mass_band(d, dx, band.data());
    for (int r = -d; r <= d; ++r) row[((r % M) + M) % M] += band[r < 0 ? -r : r];
    return row;
}

static std::vector<double> inverse_row(int d, int M, double dx)
{
    std::vector<double> band(d + 1), g(M), taps(M);
    mass_band(d, dx, band.data());
    int start = 0, n = 0;
    inverse_taps(band.data(), d, M, 0.0, g.data(), &start, &n, taps.data());
    return g;
}

template <int K>
static cudaError_t smem_optin(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(k2_sweep<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k2_sweep<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

template <int K>
static int launch_sweep2d(const Args2D &a, int grid, size_t smem, cudaStream_t s, bool pre)
{
    if (pre) k2_sweep<K, true><<<grid, 256, smem, s>>>(a);
    else k2_sweep<K><<<grid, 256, smem, s>>>(a);
    return 0;
}

extern "C" int pic2d_init(const pic2d_config *cfg, const double *x, const double *p, const double *ex,
                          const double *ey, const double *az, int32_t mem, void *stream, pic2d_handle **out)
{
    if (!cfg || !x || !p || !ex || !ey || !az || !out) return fail2d(nullptr, PIC_ERR_INVALID, "null argument");
    *out = nullptr;
    const pic2d_config &c = *cfg;
    if (!(c.L1 > 0.0) || !(c.L2 > 0.0) || c.M1 < 1 || c.M2 < 1 || (long long)c.M1 * c.M2 > kMax2DNodes ||
        c.degree < 2 || c.degree > 5 || c.np < 1 || !(c.dt > 0.0) || !(c.tol > 0.0) || c.max_iter < 1 ||
        (c.warm != 0 && c.warm != 1) ||
        !std::isfinite(c.weight) || !std::isfinite(c.hbar) || (mem != PIC_MEM_HOST && mem != PIC_MEM_DEVICE))
        return fail2d(nullptr, PIC_ERR_INVALID, "bad 2D configuration");
    pic2d_handle *h = new (std::nothrow) pic2d_handle();
    if (!h) return fail2d(nullptr, PIC_ERR_NOMEM, "handle");
    h->cfg = c;
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    h->dx1 = c.L1 / c.M1;
    h->dx2 = c.L2 / c.M2;
    h->N = c.M1 * c.M2;
    const size_t np2 = 2 * (size_t)c.np, N = (size_t)h->N;
    auto bail = [&](int rc) {
        g_err2d = h->err.empty() ? "pic2d_init failed" : h->err;
        free2d(h);
        delete h;
        return rc;
    };
    double **parts[] = {&h->x, &h->p, &h->d, &h->pk};
    for (double **a : parts)
        if (cudaMalloc((void **)a, np2 * sizeof(double)) != cudaSuccess) return bail(PIC_ERR_NOMEM);
    if (cudaMalloc((void **)&h->a0, (size_t)c.np * sizeof(double)) != cudaSuccess) return bail(PIC_ERR_NOMEM);
    double **grids[] = {&h->ex, &h->ey, &h->exk, &h->eyk, &h->ebx, &h->eby, &h->az, &h->gax, &h->gay,
                        &h->gxy, &h->gxx, &h->gyy, &h->jx, &h->jy, &h->tmp, &h->sol};
    for (double **a : grids)
        if (cudaMalloc((void **)a, N * sizeof(double)) != cudaSuccess) return bail(PIC_ERR_NOMEM);
    if (cudaMalloc((void **)&h->g1x, c.M1 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->g0x, c.M1 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->g0y, c.M2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->g1y, c.M2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->bits, 3 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&h->status, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&h->acc, 2 * sizeof(double)) != cudaSuccess)
        return bail(PIC_ERR_NOMEM);
    // positions must lie in the box
    const cudaMemcpyKind kind = mem == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (mem == PIC_MEM_HOST) {
        for (size_t a = 0; a < (size_t)c.np; ++a)
            if (!(x[2 * a] >= 0.0 && x[2 * a] < c.L1 && x[2 * a + 1] >= 0.0 && x[2 * a + 1] < c.L2) ||
                !std::isfinite(p[2 * a]) || !std::isfinite(p[2 * a + 1])) {
                fail2d(h, PIC_ERR_INVALID, "marker %zu outside the box or not finite", a);
                return bail(PIC_ERR_INVALID);
            }
    }
    if (cudaMemcpyAsync(h->x, x, np2 * sizeof(double), kind, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->p, p, np2 * sizeof(double), kind, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->ex, ex, N * sizeof(double), kind, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->ey, ey, N * sizeof(double), kind, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->az, az, N * sizeof(double), kind, h->stream) != cudaSuccess)
        return bail(fail2d(h, PIC_ERR_CUDA, "input copies"));
    // differences of A_z (host: small grids): (G_x a)_{i1,i2} = (a_{i1,i2} - a_{i1-1,i2}) / dx1,
    // (G_y a)_{i1,i2} = (a_{i1,i2} - a_{i1,i2-1}) / dx2, and the second differences of the
    // Zeeman term's quotients
    {
        std::vector<double> a(N);
        if (cudaMemcpyAsync(a.data(), h->az, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return bail(fail2d(h, PIC_ERR_CUDA, "a_z readback"));
        const std::vector<double> gx = grid_diff(a, c.M1, c.M2, 0, h->dx1), gy = grid_diff(a, c.M1, c.M2, 1, h->dx2);
        const std::vector<double> gxy = grid_diff(gy, c.M1, c.M2, 0, h->dx1);
        const std::vector<double> gxx = grid_diff(gx, c.M1, c.M2, 0, h->dx1);
        const std::vector<double> gyy = grid_diff(gy, c.M1, c.M2, 1, h->dx2);
        std::vector<double> g1x = inverse_row(c.degree - 1, c.M1, h->dx1), g0x = inverse_row(c.degree, c.M1, h->dx1);
        std::vector<double> g1y = inverse_row(c.degree - 1, c.M2, h->dx2), g0y = inverse_row(c.degree, c.M2, h->dx2);
        h->m0x = mass_row_full(c.degree, c.M1, h->dx1);
        h->m1x = mass_row_full(c.degree - 1, c.M1, h->dx1);
        h->m0y = mass_row_full(c.degree, c.M2, h->dx2);
        h->m1y = mass_row_full(c.degree - 1, c.M2, h->dx2);
        if (cudaMemcpy(h->gax, gx.data(), N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->gxy, gxy.data(), N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->gxx, gxx.data(), N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->gyy, gyy.data(), N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->gay, gy.data(), N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->g1x, g1x.data(), c.M1 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->g0x, g0x.data(), c.M1 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->g1y, g1y.data(), c.M2 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->g0y, g0y.data(), c.M2 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail2d(h, PIC_ERR_CUDA, "grid uploads"));
    }
    gauss_legendre(c.degree, h->glx, h->glw);
    const size_t smem = 2 * N * sizeof(double);
    cudaError_t e = cudaSuccess;
    switch (c.degree) {
    case 2: e = smem_optin<2>(smem); break;
    case 3: e = smem_optin<3>(smem); break;
    case 4: e = smem_optin<4>(smem); break;
    default: e = smem_optin<5>(smem); break;
    }
    if (e != cudaSuccess) return bail(fail2d(h, PIC_ERR_CUDA, "shared-memory opt-in: %s", cudaGetErrorString(e)));
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(fail2d(h, PIC_ERR_CUDA, "init sync"));
    *out = h;
    return PIC_OK;
}

static int solve_axis_pair(pic2d_handle *h, const double *ga, const double *gb, const double *in)
{
    // sol = (A_1^{-1} (x) B_2^{-1}) in: first along x2 with gb, then along x1 with ga
    const int grid = (h->N + 255) / 256;
    k2_circ<<<grid, 256, 0, h->stream>>>(h->cfg.M1, h->cfg.M2, 1, gb, in, h->tmp);
    k2_circ<<<grid, 256, 0, h->stream>>>(h->cfg.M1, h->cfg.M2, 0, ga, h->tmp, h->sol);
    CK2(cudaGetLastError());
    return PIC_OK;
}

extern "C" int pic2d_substep1(pic2d_handle *h, int32_t *iters)
{
    if (!h) return PIC_ERR_INVALID;
    const pic2d_config &c = h->cfg;
    if (c.hbar != 0.0 && !h->spin)
        return fail2d(h, PIC_ERR_INVALID, "hbar != 0: pic2d_set_spin must give the spins and b_z first");
    const size_t np2 = 2 * (size_t)c.np, N = (size_t)h->N;
    cudaStream_t s = h->stream;
    CK2(cudaMemsetAsync(h->d, 0, np2 * sizeof(double), s));
    CK2(cudaMemcpyAsync(h->pk, h->p, np2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaMemcpyAsync(h->exk, h->ex, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaMemcpyAsync(h->eyk, h->ey, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaMemcpyAsync(h->ebx, h->ex, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaMemcpyAsync(h->eby, h->ey, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    Args2D a{};
    a.M1 = c.M1; a.M2 = c.M2; a.np = c.np; a.dx1 = h->dx1; a.dx2 = h->dx2; a.dt = c.dt; a.w = c.weight;
    a.idx1 = 1.0 / h->dx1; a.idx2 = 1.0 / h->dx2; a.a0 = h->a0;
    a.x = h->x; a.pn = h->p; a.d = h->d; a.pk = h->pk;
    a.ebx = h->ebx; a.eby = h->eby; a.az = h->az; a.gax = h->gax; a.gay = h->gay;
    a.hbar = h->spin ? c.hbar : 0.0;
    a.s = h->spin; a.gxy = h->gxy; a.gxx = h->gxx; a.gyy = h->gyy; a.gbx = h->gbx; a.gby = h->gby;
    a.jx = h->jx; a.jy = h->jy; a.dmax_bits = h->bits; a.pmax_bits = h->bits + 1; a.status = h->status;
    for (int g = 0; g < 5; ++g) { a.glx[g] = h->glx[g]; a.glw[g] = h->glw[g]; }
    int num_sms = 0;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, h->device);
    const int grid = (int)std::min<long long>((c.np + 255) / 256, 4LL * (num_sms > 0 ? num_sms : 1));
    const size_t smem = 2 * N * sizeof(double);
    unsigned long long hb[3];
    int hs = 0;
    int it = 0;
    const bool warm = c.warm != 0;
    if (warm) {
        // the predicted start: delta^(0) and its current, then e^(0) = e^n - M1^{-1} j^(0)
        // and e_bar = (e^n + e^(0)) / 2 for the first sweep
        CK2(cudaMemsetAsync(h->jx, 0, N * sizeof(double), s));
        CK2(cudaMemsetAsync(h->jy, 0, N * sizeof(double), s));
        switch (c.degree) {
        case 2: launch_sweep2d<2>(a, grid, smem, s, true); break;
        case 3: launch_sweep2d<3>(a, grid, smem, s, true); break;
        case 4: launch_sweep2d<4>(a, grid, smem, s, true); break;
        default: launch_sweep2d<5>(a, grid, smem, s, true); break;
        }
        CK2(cudaGetLastError());
        int rc;
        if ((rc = solve_axis_pair(h, h->g1x, h->g0y, h->jx))) return rc;
        k2_update<<<(h->N + 255) / 256, 256, 0, s>>>(h->N, h->ex, h->sol, h->exk, h->ebx, h->bits + 2);
        if ((rc = solve_axis_pair(h, h->g0x, h->g1y, h->jy))) return rc;
        k2_update<<<(h->N + 255) / 256, 256, 0, s>>>(h->N, h->ey, h->sol, h->eyk, h->eby, h->bits + 2);
        CK2(cudaGetLastError());
    }
    for (;;) {
        CK2(cudaMemsetAsync(h->jx, 0, N * sizeof(double), s));
        CK2(cudaMemsetAsync(h->jy, 0, N * sizeof(double), s));
        CK2(cudaMemsetAsync(h->bits, 0, 3 * sizeof(unsigned long long), s));
        a.first = !warm && it == 0;          // the predicted start stored A(x^n) already
        switch (c.degree) {
        case 2: launch_sweep2d<2>(a, grid, smem, s, false); break;
        case 3: launch_sweep2d<3>(a, grid, smem, s, false); break;
        case 4: launch_sweep2d<4>(a, grid, smem, s, false); break;
        default: launch_sweep2d<5>(a, grid, smem, s, false); break;
        }
        CK2(cudaGetLastError());
        int rc;
        if ((rc = solve_axis_pair(h, h->g1x, h->g0y, h->jx))) return rc;
        k2_update<<<(h->N + 255) / 256, 256, 0, s>>>(h->N, h->ex, h->sol, h->exk, h->ebx, h->bits + 2);
        if ((rc = solve_axis_pair(h, h->g0x, h->g1y, h->jy))) return rc;
        k2_update<<<(h->N + 255) / 256, 256, 0, s>>>(h->N, h->ey, h->sol, h->eyk, h->eby, h->bits + 2);
        CK2(cudaGetLastError());
        CK2(cudaMemcpyAsync(hb, h->bits, sizeof(hb), cudaMemcpyDeviceToHost, s));
        CK2(cudaMemcpyAsync(&hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK2(cudaStreamSynchronize(s));
        ++it;
        double dm, pm, em;
        std::memcpy(&dm, &hb[0], 8);
        std::memcpy(&pm, &hb[1], 8);
        std::memcpy(&em, &hb[2], 8);
        if (hs & STATUS_NUMERIC) return fail2d(h, PIC_ERR_NUMERIC, "2D subsystem I: non-finite value or a path beyond %d cells", kMaxCross);
        if (!(dm == dm && pm == pm && em == em)) return fail2d(h, PIC_ERR_NUMERIC, "2D subsystem I: NaN increment");
        if (dm <= c.tol && pm <= c.tol && em <= c.tol) break;
        if (it >= c.max_iter) {
            if (iters) *iters = it;
            return fail2d(h, PIC_ERR_NOCONVERGE, "2D subsystem I: no convergence in %d sweeps", c.max_iter);
        }
    }
    if (iters) *iters = it;
    k2_finalize<<<(int)std::min<long long>((c.np + 255) / 256, 1024), 256, 0, s>>>(c.np, c.L1, c.L2, h->x, h->p,
                                                                                     h->d, h->pk);
    CK2(cudaMemcpyAsync(h->ex, h->exk, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaMemcpyAsync(h->ey, h->eyk, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK2(cudaGetLastError());
    CK2(cudaStreamSynchronize(s));
    return PIC_OK;
}

// e^T (A (x) B) e / 2 with circulant rows a (M1) and b (M2), on the host
static double kron_quad(const std::vector<double> &e, const std::vector<double> &ra, const std::vector<double> &rb,
                        int M1, int M2)
{
    double s = 0.0;
    for (int i1 = 0; i1 < M1; ++i1)
        for (int i2 = 0; i2 < M2; ++i2) {
            double v = 0.0;
            for (int q1 = 0; q1 < M1; ++q1) {
                const double ca = ra[((q1 - i1) % M1 + M1) % M1];
                if (ca == 0.0) continue;
                for (int q2 = 0; q2 < M2; ++q2) v += ca * rb[((q2 - i2) % M2 + M2) % M2] * e[q1 * M2 + q2];
            }
            s += e[i1 * M2 + i2] * v;
        }
    return 0.5 * s;
}

extern "C" int pic2d_energy(pic2d_handle *h, double out[4])
{
    if (!h || !out) return PIC_ERR_INVALID;
    const pic2d_config &c = h->cfg;
    CK2(cudaMemsetAsync(h->acc, 0, 2 * sizeof(double), h->stream));
    const int grid = (int)std::min<long long>((c.np + 255) / 256, 1024);
    const double hb = h->spin ? c.hbar : 0.0;
#define PIC2D_ENERGY(K)                                                                                     \
    k2_energy<K><<<grid, 256, 0, h->stream>>>(c.np, c.M1, c.M2, h->dx1, h->dx2, c.weight, h->x, h->p, h->az, hb, \
                                              h->spin, h->gax, h->gay, h->bz, h->acc)
    switch (c.degree) {
    case 2: PIC2D_ENERGY(2); break;
    case 3: PIC2D_ENERGY(3); break;
    case 4: PIC2D_ENERGY(4); break;
    default: PIC2D_ENERGY(5); break;
    }
#undef PIC2D_ENERGY
    CK2(cudaGetLastError());
    std::vector<double> ex(h->N), ey(h->N);
    double acc[2] = {0.0, 0.0};
    CK2(cudaMemcpyAsync(acc, h->acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    CK2(cudaMemcpyAsync(ex.data(), h->ex, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK2(cudaMemcpyAsync(ey.data(), h->ey, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK2(cudaStreamSynchronize(h->stream));
    const double fe = kron_quad(ex, h->m1x, h->m0y, c.M1, c.M2) + kron_quad(ey, h->m0x, h->m1y, c.M1, c.M2);
    out[0] = acc[0];
    out[1] = fe;
    out[2] = acc[1];
    out[3] = acc[0] + fe + acc[1];
    return PIC_OK;
}

extern "C" int pic2d_set_spin(pic2d_handle *h, const double *s, const double *bz, int32_t mem)
{
    if (!h || !s || !bz || (mem != PIC_MEM_HOST && mem != PIC_MEM_DEVICE)) return PIC_ERR_INVALID;
    const pic2d_config &c = h->cfg;
    const size_t N = (size_t)h->N, n3 = 3 * (size_t)c.np;
    if (!h->spin) {
        double *sp = nullptr, *b0 = nullptr, *b1 = nullptr, *b2 = nullptr;
        if (cudaMalloc((void **)&sp, n3 * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&b0, N * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&b1, N * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&b2, N * sizeof(double)) != cudaSuccess) {
            for (double *q : {sp, b0, b1, b2})
                if (q) cudaFree(q);
            return fail2d(h, PIC_ERR_NOMEM, "spin and b_z arrays");
        }
        h->spin = sp;
        h->bz = b0;
        h->gbx = b1;
        h->gby = b2;
    }
    const cudaMemcpyKind kind = mem == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    std::vector<double> b(N);
    CK2(cudaMemcpyAsync(h->spin, s, n3 * sizeof(double), kind, h->stream));
    CK2(cudaMemcpyAsync(h->bz, bz, N * sizeof(double), kind, h->stream));
    CK2(cudaMemcpyAsync(b.data(), h->bz, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK2(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < N; ++i)
        if (!std::isfinite(b[i])) return fail2d(h, PIC_ERR_INVALID, "b_z not finite at node %zu", i);
    const std::vector<double> gbx = grid_diff(b, c.M1, c.M2, 0, h->dx1), gby = grid_diff(b, c.M1, c.M2, 1, h->dx2);
    CK2(cudaMemcpyAsync(h->gbx, gbx.data(), N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK2(cudaMemcpyAsync(h->gby, gby.data(), N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK2(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

extern "C" int pic2d_get_state(pic2d_handle *h, double *x, double *p, double *ex, double *ey, int32_t mem)
{
    if (!h || (mem != PIC_MEM_HOST && mem != PIC_MEM_DEVICE)) return PIC_ERR_INVALID;
    const cudaMemcpyKind kind = mem == PIC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t np2 = 2 * (size_t)h->cfg.np, N = (size_t)h->N;
    if (x) CK2(cudaMemcpyAsync(x, h->x, np2 * sizeof(double), kind, h->stream));
    if (p) CK2(cudaMemcpyAsync(p, h->p, np2 * sizeof(double), kind, h->stream));
    if (ex) CK2(cudaMemcpyAsync(ex, h->ex, N * sizeof(double), kind, h->stream));
    if (ey) CK2(cudaMemcpyAsync(ey, h->ey, N * sizeof(double), kind, h->stream));
    CK2(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

extern "C" int pic2d_destroy(pic2d_handle *h)
{
    if (!h) return PIC_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free2d(h);
    delete h;
    return PIC_OK;
}

extern "C" const char *pic2d_last_error(const pic2d_handle *h)
{
    return h ? h->err.c_str() : g_err2d.c_str();
}
