// pic_particles.cu -- marker kernels of libpic (sm_103a).
//
// Every kernel is a persistent grid-stride loop over the structure-of-arrays
// marker state (cell int32, offset t, momentum p, iterates delta and p_new),
// read coalesced.  Field coefficients are staged once per block into shared
// memory with a periodic halo of H cells on both sides, so no index is wrapped
// in the inner loop.  Deposits are accumulated per block in double in shared
// memory and added to the global grid with one double atomic per node.
#include <climits>
#include <type_traits>

#include "pic_internal.h"

namespace pic {

template <typename R>
struct Real;
template <>
struct Real<float> { static constexpr bool fp32 = true; };
template <>
struct Real<double> { static constexpr bool fp32 = false; };

__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// Field tiles staged in shared memory, interleaved for vector loads.
template <typename R> struct FieldTile;
template <> struct FieldTile<float> {
    float2 *a;      // (a_y, a_z)
    float4 *f;      // (ebar, (G a_y), (G a_z), 0)
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
    static __host__ __device__ size_t bytes(size_t W) { return W * (sizeof(float2) + sizeof(float4)); }
};
template <> struct FieldTile<double> {
    double2 *a;     // (a_y, a_z)
    double2 *g;     // ((G a_y), (G a_z))
    double *e;      // ebar
    __device__ __forceinline__ void aa(int i, double &y, double &z) const { const double2 v = a[i]; y = v.x; z = v.y; }
    __device__ __forceinline__ void eg(int i, double &ev, double &gy, double &gz) const
    {
        const double2 v = g[i];
        ev = e[i]; gy = v.x; gz = v.y;
    }
    __device__ __forceinline__ void store(int i, double ay, double az, double ev, double gy, double gz)
    {
        a[i] = make_double2(ay, az);
        g[i] = make_double2(gy, gz);
        e[i] = ev;
    }
    static __host__ __device__ size_t bytes(size_t W) { return W * (2 * sizeof(double2) + sizeof(double)); }
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
    t.g = t.a + W;
    t.e = reinterpret_cast<double *>(t.g + W);
    return t;
}

template <typename R> __device__ __forceinline__ R fdiv_(R a, R b);
template <> __device__ __forceinline__ float fdiv_(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fdiv_(double a, double b) { return a / b; }

// Contiguous chunk of markers owned by one block (a multiple of 32, so every
// warp's lanes see consecutive, cell-sorted markers).
__device__ __forceinline__ void block_chunk(long long np, long long &beg, long long &end)
{
    long long chunk = (np + gridDim.x - 1) / gridDim.x;
    chunk = (chunk + 31) & ~31LL;
    beg = (long long)blockIdx.x * chunk;
    end = beg + chunk < np ? beg + chunk : np;
}

// ---------------------------------------------------------------------------
// Subsystem I: one Picard sweep (Sec. 4.2).  Per marker, with x^n = (c0, t0),
// the iterate x^(k) = x^n + delta^(k) and ebar = (e^n + e^(k))/2:
//   A0 = A_h(x^n), A1 = A_h(x^(k)), m = path means of Lambda^1 on x^n -> x^(k),
//   Ebar = sum m ebar, D = sum m (G a)  [= (A1-A0)/(x^(k)-x^n), exact],
//   p^(k+1) = p^n + dt Ebar - dt (A1+A0).D / (g(p^n,A1) + g(p^n,A0)),
//   delta^(k+1) = dt (p^n + p^(k+1)) / (g(p^n,A1) + g(p^(k+1),A1)) / dx,
//   j_i += w int_{x^n}^{x^n+delta^(k+1)} Lambda^1_i.
// Each block owns a contiguous chunk of the cell-sorted markers; the deposit
// goes through a per-warp register window (DepWindow), then the block's
// shared-memory row (double), then one global double atomic per touched node.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256) k_sweep1(Sweep1Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = A.H;
    const int W = A.M + 2 * H;
    double *s_acc = reinterpret_cast<double *>(smem);
    double *s_red = s_acc + W;
    FieldTile<R> F = carve_tile<R>(reinterpret_cast<unsigned char *>(s_red + 32), W);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int g = wrap_cell(i - H, A.M);
        F.store(i, A.ay[g], A.az[g], A.ebar[g], A.ga_y[g], A.ga_z[g]);
        s_acc[i] = 0.0;
    }
    __syncthreads();

    const int32_t *__restrict__ cellp = A.P.cell;
    const R *__restrict__ tp = static_cast<const R *>(A.P.t);
    const R *__restrict__ pp = static_cast<const R *>(A.P.p);
    R *__restrict__ dp = static_cast<R *>(A.P.delta);
    R *__restrict__ pnp = static_cast<R *>(A.P.pnew);
    const R dt = (R)A.dt;
    const R dtdx = (R)(A.dt / A.dx);
    const R wdx = (R)(A.w * A.dx);
    const R dlim = (R)A.Dlim;
    const R one = R(1);
    R dmax = R(0);
    bool bad = false;
    DepWindow<R, K + 4, K, K + 1, -2, 2> win;
    win.clear();
    int wb = INT_MIN;

    long long beg, end;
    block_chunk(A.np, beg, end);
    for (long long base = beg; base < end; base += blockDim.x) {
        const long long a = base + threadIdx.x;
        const bool act = a < end;
        const int c0 = act ? cellp[a] : 0;
        const int lead = __reduce_min_sync(0xffffffffu, act ? c0 : INT_MAX);
        if (lead == INT_MAX) break;                    // whole warp past the chunk end
        if (lead != wb) {
            if (wb != INT_MIN) win.flush(s_acc, wb - K - 1 + H);
            wb = lead;
        }
        if (!act) continue;
        const R t0 = tp[a];
        const R pn = pp[a];
        R v[K + 1];
        bspline_vals<K, R>(t0, v);
        R A0y = R(0), A0z = R(0);
#pragma unroll
        for (int r = 0; r <= K; ++r) {
            R y, z;
            F.aa(c0 - r + H, y, z);
            A0y += y * v[r];
            A0z += z * v[r];
        }
        const R g0 = sqrt_(one + pn * pn + A0y * A0y + A0z * A0z);
        R dold = A.warm ? fdiv_(dtdx * pn, g0) : dp[a];
        if (!(fabs(dold) <= dlim)) { bad = true; dold = R(0); }

        const R s = t0 + dold;
        const R fs = floor_(s);
        const int c1 = c0 + (int)fs;
        bspline_vals<K, R>(s - fs, v);
        R A1y = R(0), A1z = R(0);
#pragma unroll
        for (int r = 0; r <= K; ++r) {
            R y, z;
            F.aa(c1 - r + H, y, z);
            A1y += y * v[r];
            A1z += z * v[r];
        }

        R Eb = R(0), Dy = R(0), Dz = R(0);
        const R invd = (dold != R(0)) ? one / dold : R(0);
        walk_path<K, R>(t0, dold, [&](int c, R h, const R *m, bool single) {
            R e = R(0), gy = R(0), gz = R(0);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                R ev, y, z;
                F.eg(c0 + c - r + H, ev, y, z);
                e += m[r] * ev;
                gy += m[r] * y;
                gz += m[r] * z;
            }
            const R f = single ? one : h * invd;
            Eb += f * e;
            Dy += f * gy;
            Dz += f * gz;
        });

        const R q1 = one + A1y * A1y + A1z * A1z;
        const R g1 = sqrt_(q1 + pn * pn);
        const R pnew = pn + dt * Eb - dt * fdiv_((A1y + A0y) * Dy + (A1z + A0z) * Dz, g1 + g0);
        const R g2 = sqrt_(q1 + pnew * pnew);
        R dnew = fdiv_(dtdx * (pn + pnew), g1 + g2);
        if (!(fabs(dnew) <= dlim)) { bad = true; dnew = R(0); }

        walk_path<K, R>(t0, dnew, [&](int c, R h, const R *m, bool) {
            const R hw = wdx * h;
            R val[K];
#pragma unroll
            for (int r = 0; r < K; ++r) val[r] = hw * m[r];
            if (!win.put(c0 + c - wb, val)) {
#pragma unroll
                for (int r = 0; r < K; ++r) atomicAdd(&s_acc[c0 + c - r + H], (double)val[r]);
            }
        });

        R inc = fabs(dnew - dold);
        if (Real<R>::fp32) inc = inc / fmax(one, fabs(dnew));
        dmax = (inc > dmax || inc != inc) ? inc : dmax;
        dp[a] = dnew;
        pnp[a] = pnew;
    }
    if (wb != INT_MIN) win.flush(s_acc, wb - K - 1 + H);
    if (bad) atomicOr(&A.ctrl->status, STATUS_NUMERIC);
    block_max_to(&A.ctrl->dmax_bits, (double)dmax, s_red);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const double val = s_acc[i];
        if (val != 0.0) atomicAdd(&A.j[wrap_cell(i - H, A.M)], val);
    }
}

size_t sweep1_smem(int M, int H, int fp32)
{
    const size_t W = (size_t)M + 2 * (size_t)H;
    return (W + 32) * sizeof(double) + (fp32 ? FieldTile<float>::bytes(W) : FieldTile<double>::bytes(W));
}

template <typename R>
static int launch_sweep1_t(const Sweep1Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
    switch (a.K) {
    case 2: k_sweep1<2, R><<<grid, block, smem, s>>>(a); break;
    case 3: k_sweep1<3, R><<<grid, block, smem, s>>>(a); break;
    case 4: k_sweep1<4, R><<<grid, block, smem, s>>>(a); break;
    case 5: k_sweep1<5, R><<<grid, block, smem, s>>>(a); break;
    default: return 1;
    }
    return 0;
}

int launch_sweep1(const Sweep1Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
    return a.fp32 ? launch_sweep1_t<float>(a, grid, block, smem, s)
                  : launch_sweep1_t<double>(a, grid, block, smem, s);
}

// ---------------------------------------------------------------------------
// Path-integrated current of given displacements (pic_deposit CURRENT): the
// deposit half of the sweep above, in the form's precision.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256) k_current(CurrentArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = A.H;
    const int W = A.M + 2 * H;
    double *s_acc = reinterpret_cast<double *>(smem);
    for (int i = threadIdx.x; i < W; i += blockDim.x) s_acc[i] = 0.0;
    __syncthreads();
    const R *tp = static_cast<const R *>(A.P.t);
    const double wdx = A.w * A.dx;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c0 = A.P.cell[a];
        const R t0 = tp[a];
        R d = (R)(A.disp[A.P.id[a]] / A.dx);
        if (!(fabs(d) <= (R)A.Dlim)) { bad = true; continue; }
        walk_path<K, R>(t0, d, [&](int c, R h, const R *m, bool) {
            const double hw = wdx * (double)h;
#pragma unroll
            for (int r = 0; r < K; ++r) atomicAdd(&s_acc[c0 + c - r + H], hw * (double)m[r]);
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
//   s_i += w (A0 + A1) Lambda^0_i(x) / (g(p,A0) + g(p,A1))   (y and z).
// Same chunking and per-warp register windows as the subsystem-I sweep.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256) k_sweep2(Sweep2Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = A.H;
    const int W = A.M + 2 * H;
    double *s_sy = reinterpret_cast<double *>(smem);
    double *s_sz = s_sy + W;
    using R2 = typename std::conditional<std::is_same<R, float>::value, float2, double2>::type;
    R2 *s_an = reinterpret_cast<R2 *>(s_sz + W);
    R2 *s_ak = s_an + W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int g = wrap_cell(i - H, A.M);
        s_an[i].x = (R)A.an_y[g];
        s_an[i].y = (R)A.an_z[g];
        s_ak[i].x = (R)A.ak_y[g];
        s_ak[i].y = (R)A.ak_z[g];
        s_sy[i] = 0.0;
        s_sz[i] = 0.0;
    }
    __syncthreads();
    const int32_t *__restrict__ cellp = A.P.cell;
    const R *__restrict__ tp = static_cast<const R *>(A.P.t);
    const R *__restrict__ pp = static_cast<const R *>(A.P.p);
    const R w = (R)A.w;
    const R one = R(1);
    DepWindow<R, K + 3, K + 1, K + 1, -1, 1> wy, wz;
    wy.clear();
    wz.clear();
    int wb = INT_MIN;
    long long beg, end;
    block_chunk(A.np, beg, end);
    for (long long base = beg; base < end; base += blockDim.x) {
        const long long a = base + threadIdx.x;
        const bool act = a < end;
        const int c = act ? cellp[a] : 0;
        const int lead = __reduce_min_sync(0xffffffffu, act ? c : INT_MAX);
        if (lead == INT_MAX) break;
        if (lead != wb) {
            if (wb != INT_MIN) {
                wy.flush(s_sy, wb - K - 1 + H);
                wz.flush(s_sz, wb - K - 1 + H);
            }
            wb = lead;
        }
        if (!act) continue;
        const R t = tp[a];
        const R p = pp[a];
        R v[K + 1];
        bspline_vals<K, R>(t, v);
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
        const R cf = fdiv_(w, g0 + g1);
        const R fy = cf * (A0y + A1y), fz = cf * (A0z + A1z);
        R vy[K + 1], vz[K + 1];
#pragma unroll
        for (int r = 0; r <= K; ++r) {
            vy[r] = fy * v[r];
            vz[r] = fz * v[r];
        }
        if (!wy.put(c - wb, vy)) {
#pragma unroll
            for (int r = 0; r <= K; ++r) atomicAdd(&s_sy[c - r + H], (double)vy[r]);
        }
        if (!wz.put(c - wb, vz)) {
#pragma unroll
            for (int r = 0; r <= K; ++r) atomicAdd(&s_sz[c - r + H], (double)vz[r]);
        }
    }
    if (wb != INT_MIN) {
        wy.flush(s_sy, wb - K - 1 + H);
        wz.flush(s_sz, wb - K - 1 + H);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int g = wrap_cell(i - H, A.M);
        const double vy = s_sy[i], vz = s_sz[i];
        if (vy != 0.0) atomicAdd(&A.s_y[g], vy);
        if (vz != 0.0) atomicAdd(&A.s_z[g], vz);
    }
}

size_t sweep2_smem(int M, int H, int fp32)
{
    const size_t W = (size_t)M + 2 * (size_t)H;
    return 2 * W * sizeof(double) + 2 * W * (fp32 ? sizeof(float2) : sizeof(double2));
}

template <typename R>
static int launch_sweep2_t(const Sweep2Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
    switch (a.K) {
    case 2: k_sweep2<2, R><<<grid, block, smem, s>>>(a); break;
    case 3: k_sweep2<3, R><<<grid, block, smem, s>>>(a); break;
    case 4: k_sweep2<4, R><<<grid, block, smem, s>>>(a); break;
    case 5: k_sweep2<5, R><<<grid, block, smem, s>>>(a); break;
    default: return 1;
    }
    return 0;
}

int launch_sweep2(const Sweep2Args &a, int grid, int block, size_t smem, cudaStream_t s)
{
    return a.fp32 ? launch_sweep2_t<float>(a, grid, block, smem, s)
                  : launch_sweep2_t<double>(a, grid, block, smem, s);
}

// ---------------------------------------------------------------------------
// Diagnostics, evaluated in double from the stored state.
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256) k_charge(DiagArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = K + 1;
    const int W = A.M + 2 * H;
    double *s_acc = reinterpret_cast<double *>(smem);
    for (int i = threadIdx.x; i < W; i += blockDim.x) s_acc[i] = 0.0;
    __syncthreads();
    const R *tp = static_cast<const R *>(A.P.t);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const int c = A.P.cell[a];
        double v[K + 1];
        bspline_vals<K, double>((double)tp[a], v);
#pragma unroll
        for (int r = 0; r <= K; ++r) atomicAdd(&s_acc[c - r + H], A.w * v[r]);
    }
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
// wrapped periodically), p^{n+1} = p^(k+1); the iterate is reset.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_finalize1(long long np, int M, PartPtrs P)
{
    R *tp = static_cast<R *>(P.t);
    R *pp = static_cast<R *>(P.p);
    R *dp = static_cast<R *>(P.delta);
    const R *pnp = static_cast<const R *>(P.pnew);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < np; a += stride) {
        const R s = tp[a] + dp[a];
        const R f = floor_(s);
        int c = P.cell[a] + (int)f;
        R t = s - f;
        if (t >= R(1)) { t -= R(1); c += 1; }
        P.cell[a] = wrap_cell(c, M);
        tp[a] = t;
        pp[a] = pnp[a];
        dp[a] = R(0);
    }
}

int launch_finalize1(int fp32, long long np, int M, PartPtrs P, int grid, int block, cudaStream_t s)
{
    if (fp32) k_finalize1<float><<<grid, block, 0, s>>>(np, M, P);
    else k_finalize1<double><<<grid, block, 0, s>>>(np, M, P);
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
        P.id[a] = a;
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

// ---------------------------------------------------------------------------
// Counting sort of the markers by cell (between steps; delta = 0, p_new = p).
// counts: 2*M int32 scratch (histogram, then cursors).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_hist(long long np, int M, const int32_t *cell, int32_t *counts)
{
    extern __shared__ int32_t s_h[];
    for (int i = threadIdx.x; i < M; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < np; a += stride)
        atomicAdd(&s_h[cell[a]], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x)
        if (s_h[i]) atomicAdd(&counts[i], s_h[i]);
}

__global__ void k_scan(int M, int32_t *counts)
{
    // exclusive scan of M counts into cursors (single block; M <= 8192)
    __shared__ long long s_part[1024];
    const int per = (M + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(M, lo + per);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    s_part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) { long long v = s_part[i]; s_part[i] = run; run += v; }
    }
    __syncthreads();
    long long run = s_part[threadIdx.x];
    for (int i = lo; i < hi; ++i) { const int v = counts[i]; counts[M + i] = (int32_t)run; run += v; }
}

template <typename R>
__global__ void __launch_bounds__(256) k_scatter(long long np, int M, PartPtrs S, PartPtrs D, int32_t *cursor)
{
    const R *ts = static_cast<const R *>(S.t);
    const R *ps = static_cast<const R *>(S.p);
    R *td = static_cast<R *>(D.t);
    R *pd = static_cast<R *>(D.p);
    R *pnd = static_cast<R *>(D.pnew);
    R *dd = static_cast<R *>(D.delta);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < np; a += stride) {
        const int c = S.cell[a];
        const long long j = atomicAdd(&cursor[c], 1);
        D.cell[j] = c;
        td[j] = ts[a];
        const R p = ps[a];
        pd[j] = p;
        pnd[j] = p;
        dd[j] = R(0);
        D.id[j] = S.id[a];
    }
}

int launch_sort(int fp32, long long np, int M, PartPtrs src, PartPtrs dst, int32_t *counts,
                int grid, int block, cudaStream_t s)
{
    if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * (size_t)M, s) != cudaSuccess) return 1;
    k_hist<<<grid, block, sizeof(int32_t) * M, s>>>(np, M, src.cell, counts);
    k_scan<<<1, 1024, 0, s>>>(M, counts);
    if (fp32) k_scatter<float><<<grid, block, 0, s>>>(np, M, src, dst, counts + M);
    else k_scatter<double><<<grid, block, 0, s>>>(np, M, src, dst, counts + M);
    return 0;
}


// ---------------------------------------------------------------------------
// Dynamic shared-memory opt-in (per kernel instantiation) and occupancy.
// ---------------------------------------------------------------------------
template <int K, typename R>
static int set_attrs_kr(size_t s1, size_t s2, size_t s3)
{
    if (cudaFuncSetAttribute(k_sweep1<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) return 1;
    if (cudaFuncSetAttribute(k_sweep2<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2)) return 1;
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

int sweep_blocks_per_sm(int K, int fp32, int which, int block, size_t smem)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define OCC(KK, RR)                                                                                  \
    if (K == KK && (fp32 != 0) == std::is_same<RR, float>::value)                                    \
        e = which == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep1<KK, RR>, block, smem) \
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<KK, RR>, block, smem);
    OCC(2, float) OCC(3, float) OCC(4, float) OCC(5, float)
    OCC(2, double) OCC(3, double) OCC(4, double) OCC(5, double)
#undef OCC
    return e == cudaSuccess ? n : 0;
}

}  // namespace pic

int pic_set_smem_attrs(size_t s1, size_t s2, size_t s3)
{
    return pic::set_attrs_r<float>(s1, s2, s3) | pic::set_attrs_r<double>(s1, s2, s3);
}

namespace pic {
}  // namespace pic
