// pic_mlp.cu -- the learned warm start of the subsystem-I fixed point.
//
// A small network proposes each marker's displacement x^(0) - x^n for the
// implicit substep of subsystem I (Sec. 4.2); the Picard iteration then runs to
// the same tolerance, so the proposal changes only the number of sweeps, never
// the converged state or the conservation properties.
//
// Network: 6 inputs (cell-relative x, p, E_x(x^n), A_y(x^n), A_z(x^n), dt), each
// normalised by (v - shift) * scale; three hidden layers of width 64 with GELU
// (tanh form); 2 outputs, scaled by out_scale, read as
//   y0 = (x^{n+1} - x^n - dt p/gamma(p, A(x^n))) / dt^2   (residual of the explicit predictor)
//   y1 = (p^{n+1} - p^n - dt E_x(x^n)) / dt^2.
// Parameters: one float vector W1 (64x6, row-major [out][in]), b1, W2 (64x64),
// b2, W3, b3, W4 (2x64), b4 -- 8898 numbers.
//
// Inference runs on the tensor cores: bf16 operands, fp32 accumulation, with
// mma.sync m16n8k16 (a warp computes 32 markers as two 16-row tiles that share
// every weight fragment; the fp32 accumulator fragment of one layer passes
// through the GELU in packed bf16 and becomes the bf16 A fragment of the next, in
// registers).  Training (forward + backward + Adam) runs in fp32 on the CUDA cores.
#include <cuda_bf16.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "pic.h"
#include "pic_internal.h"

namespace pic {

constexpr int kIn = 6, kHid = 64, kOut = 2;
constexpr int kNParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;   // 8898
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid,
              kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kOut * kHid;
static_assert(kOffB4 + kOut == kNParams, "parameter packing");
constexpr int kNorm = 2 * kIn + kOut;     // shift[6], scale[6], out_scale[2]

// shared-memory image of the network for the tensor-core path (bf16 rows padded
// so that the 8 rows a B fragment touches fall in distinct banks)
constexpr int kS1 = 24, kS = 72;
struct MlpTC {
    __nv_bfloat16 W1[kHid * kS1];
    __nv_bfloat16 W2[kHid * kS];
    __nv_bfloat16 W3[kHid * kS];
    __nv_bfloat16 W4[8 * kS];
    float b1[kHid], b2[kHid], b3[kHid], b4[8];
    float norm[kNorm];
};

__device__ __forceinline__ float gelu_exact(float z)
{
    return 0.5f * z * (1.f + tanhf(0.7978845608028654f * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
    const float t = tanhf(u);
    const float du = 0.7978845608028654f * (1.f + 3.f * 0.044715f * z * z);
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * du;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

// GELU (tanh form) of two pre-activations, evaluated in packed bf16 arithmetic on
// their bf16 roundings and returned packed: the result is a bf16 activation of
// the next layer either way, and one tanh.approx.bf16x2 serves both values.
__device__ __forceinline__ uint32_t gelu_bf16x2(float z0, float z1)
{
    const __nv_bfloat162 z = __floats2bfloat162_rn(z0, z1);
    const __nv_bfloat162 c0 = __float2bfloat162_rn(0.7978845608028654f);
    const __nv_bfloat162 c1 = __float2bfloat162_rn(0.7978845608028654f * 0.044715f);
    const __nv_bfloat162 half = __float2bfloat162_rn(0.5f);
    const __nv_bfloat162 u = __hmul2(z, __hfma2(__hmul2(z, z), c1, c0));   // c0 z + c1 z^3
    uint32_t ui, ti;
    memcpy(&ui, &u, 4);
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(ti) : "r"(ui));
    __nv_bfloat162 th;
    memcpy(&th, &ti, 4);
    const __nv_bfloat162 out = __hmul2(z, __hfma2(th, half, half));         // z (1 + tanh u) / 2
    uint32_t o;
    memcpy(&o, &out, 4);
    return o;
}

// four 8x8 bf16 matrices from shared memory; lane l supplies the row address of
// matrix l / 8, row l % 8
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage the network from fp32 parameters (global) into the shared image.
__device__ void stage_tc(MlpTC &S, const float *params, const float *norm)
{
    for (int i = threadIdx.x; i < kHid * kS1; i += blockDim.x) {
        const int n = i / kS1, k = i % kS1;
        S.W1[i] = __float2bfloat16(k < kIn ? params[kOffW1 + n * kIn + k] : 0.f);
    }
    for (int i = threadIdx.x; i < kHid * kS; i += blockDim.x) {
        const int n = i / kS, k = i % kS;
        S.W2[i] = __float2bfloat16(k < kHid ? params[kOffW2 + n * kHid + k] : 0.f);
        S.W3[i] = __float2bfloat16(k < kHid ? params[kOffW3 + n * kHid + k] : 0.f);
    }
    for (int i = threadIdx.x; i < 8 * kS; i += blockDim.x) {
        const int n = i / kS, k = i % kS;
        S.W4[i] = __float2bfloat16(n < kOut && k < kHid ? params[kOffW4 + n * kHid + k] : 0.f);
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        S.b1[i] = params[kOffB1 + i];
        S.b2[i] = params[kOffB2 + i];
        S.b3[i] = params[kOffB3 + i];
    }
    if (threadIdx.x < 8) S.b4[threadIdx.x] = threadIdx.x < kOut ? params[kOffB4 + threadIdx.x] : 0.f;
    if (threadIdx.x < kNorm) S.norm[threadIdx.x] = norm[threadIdx.x];
}

// One hidden layer for the warp's two 16-row tiles: D (16 x 64 each) =
// act(A (16 x 16*KT) W^T + b), re-packed as the bf16 A fragments of the next
// layer (4 k-tiles).  W is [n][k] row-major in shared memory; each ldmatrix.x4
// brings the B fragments of two n-tiles at one k-tile, used by both row tiles.
template <int KT>
__device__ __forceinline__ void hidden_layer2(const uint32_t (&a)[2][KT][4], const __nv_bfloat16 *W, int stride,
                                              const float *b, uint32_t (&out)[2][4][4])
{
    const int lane = threadIdx.x & 31, q = lane & 3;
    const int mi = lane >> 3, rr = lane & 7;
#pragma unroll
    for (int np2 = 0; np2 < 4; ++np2) {           // n-tiles 2 np2, 2 np2 + 1
        float d[2][2][4];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float b0 = b[16 * np2 + 8 * s + 2 * q], b1 = b[16 * np2 + 8 * s + 2 * q + 1];
#pragma unroll
            for (int tile = 0; tile < 2; ++tile) {
                d[tile][s][0] = b0; d[tile][s][1] = b1; d[tile][s][2] = b0; d[tile][s][3] = b1;
            }
        }
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            uint32_t bf[4];
            // matrices: (n-tile 2np2, k lo), (2np2, k hi), (2np2+1, k lo), (2np2+1, k hi)
            ldsm_x4(bf, W + (16 * np2 + 8 * (mi >> 1) + rr) * stride + 16 * kt + 8 * (mi & 1));
#pragma unroll
            for (int tile = 0; tile < 2; ++tile) {
                mma_bf16(d[tile][0], a[tile][kt], bf[0], bf[1]);
                mma_bf16(d[tile][1], a[tile][kt], bf[2], bf[3]);
            }
        }
#pragma unroll
        for (int tile = 0; tile < 2; ++tile) {
            out[tile][np2][0] = gelu_bf16x2(d[tile][0][0], d[tile][0][1]);
            out[tile][np2][1] = gelu_bf16x2(d[tile][0][2], d[tile][0][3]);
            out[tile][np2][2] = gelu_bf16x2(d[tile][1][0], d[tile][1][1]);
            out[tile][np2][3] = gelu_bf16x2(d[tile][1][2], d[tile][1][3]);
        }
    }
}

// 32 markers (two 16-row tiles) through the network.  X: 32 rows of 16 bf16
// (normalised features, zero padded) at row stride xs.  On return lanes with
// q == 0 hold, for tile t, the outputs of rows g (y[t][0..1]) and g + 8 (y[t][2..3]).
__device__ __forceinline__ void mlp_tile32(const MlpTC &S, const __nv_bfloat16 *X, int xs, float (&y)[2][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    uint32_t a0[2][1][4];
#pragma unroll
    for (int tile = 0; tile < 2; ++tile) {
        const __nv_bfloat16 *Xt = X + tile * 16 * xs;
        a0[tile][0][0] = *reinterpret_cast<const uint32_t *>(Xt + g * xs + 2 * q);
        a0[tile][0][1] = *reinterpret_cast<const uint32_t *>(Xt + (g + 8) * xs + 2 * q);
        a0[tile][0][2] = *reinterpret_cast<const uint32_t *>(Xt + g * xs + 2 * q + 8);
        a0[tile][0][3] = *reinterpret_cast<const uint32_t *>(Xt + (g + 8) * xs + 2 * q + 8);
    }
    uint32_t h1[2][4][4], h2[2][4][4];
    hidden_layer2<1>(a0, S.W1, kS1, S.b1, h1);
    hidden_layer2<4>(h1, S.W2, kS, S.b2, h2);
    hidden_layer2<4>(h2, S.W3, kS, S.b3, h1);
#pragma unroll
    for (int tile = 0; tile < 2; ++tile) {
        float d[4];
        d[0] = S.b4[2 * q]; d[1] = S.b4[2 * q + 1]; d[2] = d[0]; d[3] = d[1];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const __nv_bfloat16 *row = S.W4 + g * kS + 16 * kt + 2 * q;
            mma_bf16(d, h1[tile][kt], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
        y[tile][0] = d[0]; y[tile][1] = d[1]; y[tile][2] = d[2]; y[tile][3] = d[3];
    }
}

// Per-warp staging of 32 markers' features and outputs.
constexpr int kXS = 24;   // bf16 row stride of the feature tile (16 used, 16-byte aligned rows)
struct WarpTile {
    __nv_bfloat16 X[32 * kXS];
    float Y[32][2];
};

// Zero the padding columns of the warp tile once; rows then take only their
// six features.
__device__ __forceinline__ void clear_tile(WarpTile &T)
{
    const int lane = threadIdx.x & 31;
    uint32_t *w = reinterpret_cast<uint32_t *>(T.X);
    for (int i = lane; i < 32 * kXS / 2; i += 32) w[i] = 0u;
    __syncwarp();
}

// Features of one marker into row r of the warp tile, normalised (columns 0..5).
__device__ __forceinline__ void put_features(WarpTile &T, const float *norm, int r, const float f[kIn])
{
    uint32_t *row = reinterpret_cast<uint32_t *>(T.X + r * kXS);
#pragma unroll
    for (int i = 0; i < kIn / 2; ++i)
        row[i] = pack_bf16((f[2 * i] - norm[2 * i]) * norm[kIn + 2 * i],
                           (f[2 * i + 1] - norm[2 * i + 1]) * norm[kIn + 2 * i + 1]);
}

// Run the warp's 32 rows (two 16-row tiles) and leave the scaled outputs in T.Y.
__device__ __forceinline__ void run_warp_tile(const MlpTC &S, WarpTile &T)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    __syncwarp();
    float y[2][4];
    mlp_tile32(S, T.X, kXS, y);
    if (q == 0) {
#pragma unroll
        for (int tile = 0; tile < 2; ++tile) {
            T.Y[tile * 16 + g][0] = y[tile][0] * S.norm[2 * kIn];
            T.Y[tile * 16 + g][1] = y[tile][1] * S.norm[2 * kIn + 1];
            T.Y[tile * 16 + g + 8][0] = y[tile][2] * S.norm[2 * kIn];
            T.Y[tile * 16 + g + 8][1] = y[tile][3] * S.norm[2 * kIn + 1];
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Standalone inference: X (B x 6 raw features, fp32) -> Y (B x 2 scaled outputs).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_mlp_infer(const float *params, const float *norm, const float *X,
                                                   long long B, float *Y)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpTC &S = *reinterpret_cast<MlpTC *>(smem);
    WarpTile *tiles = reinterpret_cast<WarpTile *>(smem + ((sizeof(MlpTC) + 15) & ~size_t(15)));
    stage_tc(S, params, norm);
    __syncthreads();
    WarpTile &T = tiles[threadIdx.x >> 5];
    clear_tile(T);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < B; base += stride) {
        const long long a = base + lane;
        float f[kIn];
#pragma unroll
        for (int i = 0; i < kIn; ++i) f[i] = a < B ? X[a * kIn + i] : S.norm[i];
        put_features(T, S.norm, lane, f);
        run_warp_tile(S, T);
        if (a < B) {
            Y[2 * a] = T.Y[lane][0];
            Y[2 * a + 1] = T.Y[lane][1];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Warm start of subsystem I: delta^(0) = tau p/g0 + y0 dt^2/dx for every marker,
// with the features gathered at x^n from e_x^n and a^n (staged in shared memory).
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(256, 2) k_warm_mlp(WarmArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpTC &S = *reinterpret_cast<MlpTC *>(smem);
    unsigned char *p = smem + ((sizeof(MlpTC) + 15) & ~size_t(15));
    WarpTile *tiles = reinterpret_cast<WarpTile *>(p);
    p += sizeof(WarpTile) * (blockDim.x >> 5);
    const int H = K + 1;
    const int W = A.M + 2 * H;
    float *s_e = reinterpret_cast<float *>(p);
    float2 *s_a = reinterpret_cast<float2 *>(s_e + ((W + 1) & ~1));
    stage_tc(S, A.params, A.norm);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int g = wrap_cell(i - H, A.M);
        s_e[i] = (float)A.ex[g];
        s_a[i] = make_float2((float)A.ay[g], (float)A.az[g]);
    }
    __syncthreads();
    WarpTile &T = tiles[threadIdx.x >> 5];
    clear_tile(T);
    const int lane = threadIdx.x & 31;
    const R *tp = static_cast<const R *>(A.P.t);
    const R *pp = static_cast<const R *>(A.P.p);
    R *dp = static_cast<R *>(A.P.delta);
    const float tau = (float)(A.dt / A.dx);
    const float c2 = (float)(A.dt * A.dt / A.dx);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < A.np; base += stride) {
        const long long a = base + lane;
        const bool act = a < A.np;
        float f[kIn], pn = 0.f, g0 = 1.f;
        if (act) {
            const int c = A.P.cell[a];
            const float t = (float)tp[a];
            pn = (float)pp[a];
            float v[K + 1], u[K];
            bspline_vals<K, float>(t, v);
            bspline_vals<K - 1, float>(t, u);
            float Ay = 0.f, Az = 0.f, Ex = 0.f;
#pragma unroll
            for (int r = 0; r <= K; ++r) {
                const float2 av = s_a[c - r + H];
                Ay += av.x * v[r];
                Az += av.y * v[r];
            }
#pragma unroll
            for (int r = 0; r < K; ++r) Ex += s_e[c - r + H] * u[r];
            g0 = sqrtf(1.f + pn * pn + Ay * Ay + Az * Az);
            f[0] = t; f[1] = pn; f[2] = Ex; f[3] = Ay; f[4] = Az; f[5] = (float)A.dt;
        } else {
#pragma unroll
            for (int i = 0; i < kIn; ++i) f[i] = S.norm[i];
        }
        put_features(T, S.norm, lane, f);
        run_warp_tile(S, T);
        if (act) dp[a] = (R)(tau * pn / g0 + T.Y[lane][0] * c2);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Training: loss = mean over the batch of sum_o (y_o - T_o / out_scale_o)^2 on
// the normalised outputs; gradients by the chain rule in fp32 (exact tanh).
// One block takes 32 samples; weight gradients are summed in shared memory and
// added to the global gradient once per block.
// ---------------------------------------------------------------------------
constexpr int kTB = 32;
struct TrainSmem {
    float Wt[kNParams];
    float G[kNParams];
    float h0[kTB][kIn];
    float z1[kTB][kHid], h1[kTB][kHid], z2[kTB][kHid], h2[kTB][kHid], z3[kTB][kHid], h3[kTB][kHid];
    float y[kTB][kOut];
    float d1[kTB][kHid], d2[kTB][kHid];
};

__device__ __forceinline__ void dense_fwd(const float *W, const float *b, const float *hin, int nin,
                                          float (*z)[kHid], float (*h)[kHid], int ns)
{
    for (int i = threadIdx.x; i < ns * kHid; i += blockDim.x) {
        const int s = i / kHid, n = i % kHid;
        float acc = b[n];
        for (int k = 0; k < nin; ++k) acc += W[n * nin + k] * hin[s * nin + k];
        z[s][n] = acc;
        h[s][n] = gelu_exact(acc);
    }
}

__global__ void __launch_bounds__(256) k_mlp_train(const float *params, const float *norm, const float *X,
                                                   const float *Tg, long long B, float *grad, double *loss)
{
    extern __shared__ __align__(16) unsigned char smem[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem);
    const long long s0 = (long long)blockIdx.x * kTB;
    const int ns = (int)min((long long)kTB, B - s0);
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) {
        S.Wt[i] = params[i];
        S.G[i] = 0.f;
    }
    for (int i = threadIdx.x; i < ns * kIn; i += blockDim.x) {
        const int s = i / kIn, k = i % kIn;
        S.h0[s][k] = (X[(s0 + s) * kIn + k] - norm[k]) * norm[kIn + k];
    }
    __syncthreads();
    dense_fwd(S.Wt + kOffW1, S.Wt + kOffB1, &S.h0[0][0], kIn, S.z1, S.h1, ns);
    __syncthreads();
    dense_fwd(S.Wt + kOffW2, S.Wt + kOffB2, &S.h1[0][0], kHid, S.z2, S.h2, ns);
    __syncthreads();
    dense_fwd(S.Wt + kOffW3, S.Wt + kOffB3, &S.h2[0][0], kHid, S.z3, S.h3, ns);
    __syncthreads();
    // output layer and dL/dy
    if (threadIdx.x < ns * kOut) {
        const int s = threadIdx.x / kOut, o = threadIdx.x % kOut;
        float acc = S.Wt[kOffB4 + o];
        for (int k = 0; k < kHid; ++k) acc += S.Wt[kOffW4 + o * kHid + k] * S.h3[s][k];
        const float r = acc - Tg[(s0 + s) * kOut + o] / norm[2 * kIn + o];
        S.y[s][o] = 2.f * r / (float)B;
        atomicAdd(loss, (double)r * (double)r / (double)B);
    }
    __syncthreads();
    // W4, b4
    for (int i = threadIdx.x; i < kOut * kHid; i += blockDim.x) {
        const int o = i / kHid, k = i % kHid;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += S.y[s][o] * S.h3[s][k];
        S.G[kOffW4 + i] += acc;
    }
    if (threadIdx.x < kOut) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += S.y[s][threadIdx.x];
        S.G[kOffB4 + threadIdx.x] += acc;
    }
    // d3 = (dY W4) * gelu'(z3)   (into d1)
    for (int i = threadIdx.x; i < ns * kHid; i += blockDim.x) {
        const int s = i / kHid, k = i % kHid;
        float acc = 0.f;
        for (int o = 0; o < kOut; ++o) acc += S.y[s][o] * S.Wt[kOffW4 + o * kHid + k];
        S.d1[s][k] = acc * gelu_grad(S.z3[s][k]);
    }
    __syncthreads();
    // hidden layers 3, 2, 1 (d in, gradient of W/b, d out)
    float(*din)[kHid] = S.d1;
    float(*dout)[kHid] = S.d2;
    const float(*hprev[3])[kHid] = {S.h2, S.h1, nullptr};
    const float(*zprev[3])[kHid] = {S.z2, S.z1, nullptr};
    const int offW[3] = {kOffW3, kOffW2, kOffW1}, offB[3] = {kOffB3, kOffB2, kOffB1};
    for (int L = 0; L < 3; ++L) {
        const int nin = (L == 2) ? kIn : kHid;
        for (int i = threadIdx.x; i < kHid * nin; i += blockDim.x) {
            const int n = i / nin, k = i % nin;
            float acc = 0.f;
            if (L == 2)
                for (int s = 0; s < ns; ++s) acc += din[s][n] * S.h0[s][k];
            else
                for (int s = 0; s < ns; ++s) acc += din[s][n] * hprev[L][s][k];
            S.G[offW[L] + i] += acc;
        }
        for (int n = threadIdx.x; n < kHid; n += blockDim.x) {
            float acc = 0.f;
            for (int s = 0; s < ns; ++s) acc += din[s][n];
            S.G[offB[L] + n] += acc;
        }
        if (L < 2) {
            for (int i = threadIdx.x; i < ns * kHid; i += blockDim.x) {
                const int s = i / kHid, k = i % kHid;
                float acc = 0.f;
                for (int n = 0; n < kHid; ++n) acc += din[s][n] * S.Wt[offW[L] + n * kHid + k];
                dout[s][k] = acc * gelu_grad(zprev[L][s][k]);
            }
        }
        __syncthreads();
        float(*tmp)[kHid] = din;
        din = dout;
        dout = tmp;
    }
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) atomicAdd(&grad[i], S.G[i]);
}

__global__ void k_adam(float *params, float *m, float *v, const float *g, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t mlp_infer_smem(int warps) { return ((sizeof(MlpTC) + 15) & ~size_t(15)) + sizeof(WarpTile) * warps; }

size_t warm_mlp_smem(int M, int K, int warps)
{
    const size_t W = (size_t)M + 2 * (size_t)(K + 1);
    return mlp_infer_smem(warps) + ((W + 1) & ~size_t(1)) * sizeof(float) + W * sizeof(float2);
}

int launch_warm_mlp(const WarmArgs &a, int grid, cudaStream_t s)
{
    const int block = 256;
    const size_t smem = warm_mlp_smem(a.M, a.K, block / 32);
    static size_t opted = 0;
    if (smem > opted) {
        cudaError_t e = cudaSuccess;
#define ATTR(KK, RR) e = e ? e : cudaFuncSetAttribute(k_warm_mlp<KK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        ATTR(2, float) ATTR(3, float) ATTR(4, float) ATTR(5, float)
        ATTR(2, double) ATTR(3, double) ATTR(4, double) ATTR(5, double)
#undef ATTR
        if (e != cudaSuccess) return 1;
        opted = smem;
    }
#define LAUNCH(KK)                                                                               \
    case KK:                                                                                     \
        if (a.fp32) k_warm_mlp<KK, float><<<grid, block, smem, s>>>(a);                          \
        else k_warm_mlp<KK, double><<<grid, block, smem, s>>>(a);                                \
        break;
    switch (a.K) {
        LAUNCH(2) LAUNCH(3) LAUNCH(4) LAUNCH(5)
    default: return 1;
    }
#undef LAUNCH
    return 0;
}

}  // namespace pic

using namespace pic;

struct pic_mlp {
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    float *params = nullptr, *norm = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    double *loss = nullptr;
    long long t = 0;
};

static int mlp_fail(int code, const char *msg)
{
    set_thread_error(msg);
    return code;
}

extern "C" int pic_mlp_create(const float *params, const float *norm, void *stream, pic_mlp **out)
{
    if (!out || !norm) return mlp_fail(PIC_ERR_INVALID, "pic_mlp_create: out and norm are required");
    *out = nullptr;
    pic_mlp *m = new (std::nothrow) pic_mlp();
    if (!m) return PIC_ERR_NOMEM;
    m->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
    bool ok = cudaMalloc((void **)&m->params, kNParams * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&m->norm, kNorm * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&m->grad, kNParams * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&m->m, kNParams * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&m->v, kNParams * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&m->loss, sizeof(double)) == cudaSuccess;
    if (!ok) {
        pic_mlp_destroy(m);
        return mlp_fail(PIC_ERR_NOMEM, "pic_mlp_create: cudaMalloc failed");
    }
    std::vector<float> zero(kNParams, 0.f);
    cudaMemcpyAsync(m->params, params ? params : zero.data(), kNParams * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->norm, norm, kNorm * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->m, 0, kNParams * sizeof(float), m->stream);
    cudaMemsetAsync(m->v, 0, kNParams * sizeof(float), m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        pic_mlp_destroy(m);
        return mlp_fail(PIC_ERR_CUDA, "pic_mlp_create: upload failed");
    }
    *out = m;
    return PIC_OK;
}

extern "C" int pic_mlp_destroy(pic_mlp *m)
{
    if (!m) return PIC_OK;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->params); cudaFree(m->norm); cudaFree(m->grad); cudaFree(m->m); cudaFree(m->v); cudaFree(m->loss);
    delete m;
    return PIC_OK;
}

extern "C" int pic_mlp_get_params(pic_mlp *m, float *params_host)
{
    if (!m || !params_host) return mlp_fail(PIC_ERR_INVALID, "pic_mlp_get_params: null argument");
    if (cudaMemcpyAsync(params_host, m->params, kNParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream) ||
        cudaStreamSynchronize(m->stream))
        return mlp_fail(PIC_ERR_CUDA, "pic_mlp_get_params: copy failed");
    return PIC_OK;
}

extern "C" int pic_mlp_grad(pic_mlp *m, const float *X, const float *T, int64_t B, float *grad_out, double *loss_out)
{
    if (!m || !X || !T || B < 1) return mlp_fail(PIC_ERR_INVALID, "pic_mlp_grad: invalid argument");
    static bool opted = false;
    if (!opted) {
        if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)))
            return mlp_fail(PIC_ERR_CUDA, "pic_mlp_grad: shared-memory opt-in failed");
        opted = true;
    }
    cudaMemsetAsync(m->grad, 0, kNParams * sizeof(float), m->stream);
    cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
    const long long nblk = (B + kTB - 1) / kTB;
    k_mlp_train<<<(unsigned)nblk, 256, sizeof(TrainSmem), m->stream>>>(m->params, m->norm, X, T, B, m->grad, m->loss);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(PIC_ERR_CUDA, "pic_mlp_grad: launch failed");
    if (grad_out && cudaMemcpyAsync(grad_out, m->grad, kNParams * sizeof(float), cudaMemcpyDeviceToDevice, m->stream))
        return mlp_fail(PIC_ERR_CUDA, "pic_mlp_grad: copy failed");
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) ||
            cudaStreamSynchronize(m->stream))
            return mlp_fail(PIC_ERR_CUDA, "pic_mlp_grad: loss copy failed");
    }
    return PIC_OK;
}

extern "C" int pic_mlp_train_step(pic_mlp *m, const float *X, const float *T, int64_t B, float lr, double *loss_out)
{
    int rc = pic_mlp_grad(m, X, T, B, nullptr, nullptr);
    if (rc) return rc;
    m->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
    k_adam<<<(kNParams + 255) / 256, 256, 0, m->stream>>>(m->params, m->m, m->v, m->grad, kNParams, lr, b1, b2,
                                                         1e-8f, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(PIC_ERR_CUDA, "pic_mlp_train_step: launch failed");
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) ||
            cudaStreamSynchronize(m->stream))
            return mlp_fail(PIC_ERR_CUDA, "pic_mlp_train_step: loss copy failed");
    }
    return PIC_OK;
}

extern "C" int pic_mlp_infer(pic_mlp *m, const float *X, int64_t B, float *Y)
{
    if (!m || !X || !Y || B < 0) return mlp_fail(PIC_ERR_INVALID, "pic_mlp_infer: invalid argument");
    if (B == 0) return PIC_OK;
    const int block = 256;
    const size_t smem = mlp_infer_smem(block / 32);
    static bool opted = false;
    if (!opted) {
        if (cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return mlp_fail(PIC_ERR_CUDA, "pic_mlp_infer: shared-memory opt-in failed");
        opted = true;
    }
    long long blocks = (B + block - 1) / block;
    if (blocks > (long long)m->num_sms * 4) blocks = (long long)m->num_sms * 4;
    k_mlp_infer<<<(unsigned)blocks, block, smem, m->stream>>>(m->params, m->norm, X, B, Y);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mlp_fail(PIC_ERR_CUDA, "pic_mlp_infer: kernel failed");
    return PIC_OK;
}

// accessors for the handle code (pic_api.cu)
const float *mlp_params(const pic_mlp *m) { return m->params; }
const float *mlp_norm(const pic_mlp *m) { return m->norm; }
