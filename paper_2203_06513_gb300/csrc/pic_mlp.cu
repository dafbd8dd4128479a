// pic_mlp.cu -- the learned warm start of the subsystem-I fixed point.
//
// A small network proposes each marker's displacement x^(0) - x^n for the
// implicit substep of subsystem I (Sec. 4.2); the Picard iteration then runs to
// the same tolerance, so the proposal changes only the number of sweeps, never
// the converged state or the conservation properties.
//
// Network: 6 inputs (cell-relative x, p, E_x(x^n), A_y(x^n), A_z(x^n), dt), each
// normalised by (v - shift) * scale; three hidden layers of width 64 with ReLU;
// 2 outputs, scaled by out_scale, read as
//   y0 = (x^{n+1} - x^n - dt p/gamma(p, A(x^n))) / dt^2   (residual of the explicit predictor)
//   y1 = (p^{n+1} - p^n - dt E_x(x^n)) / dt^2.
// Parameters: one float vector W1 (64x6, row-major [out][in]), b1, W2 (64x64),
// b2, W3, b3, W4 (2x64), b4 -- 8898 numbers.
//
// Inference runs on the 5th-generation tensor cores (tcgen05.mma, bf16 operands
// in shared memory, fp32 accumulators in tensor memory), 128 markers per tile;
// the ReLU runs in packed bf16 on each thread's accumulator row.  Training
// (forward + backward + Adam) runs in fp32 on the CUDA cores.
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

__device__ __forceinline__ float relu(float z) { return fmaxf(z, 0.f); }

// derivative of the ReLU, taken as 0 at z = 0
__device__ __forceinline__ float relu_grad(float z) { return z > 0.f ? 1.f : 0.f; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

// ReLU of two pre-activations, rounded to bf16 and packed: one packed max a pair.
__device__ __forceinline__ uint32_t relu_bf16x2(float z0, float z1)
{
    const __nv_bfloat162 out = __hmax2(__floats2bfloat162_rn(z0, z1), __float2bfloat162_rn(0.f));
    uint32_t o;
    memcpy(&o, &out, 4);
    return o;
}

// ---------------------------------------------------------------------------
// Tensor-core inference with tcgen05 (5th-generation tensor cores, accumulators
// in tensor memory).  One block of 1024 threads per SM runs 8 independent chains,
// one per warpgroup; a chain takes 128 markers at a time, one row per thread.  Per
// layer the chain writes its rows' bf16 activations to shared memory in the
// canonical K-major layout (8-row x 16-byte core matrices), one of its threads
// issues the layer's tcgen05.mma instructions (M = 128, N = 64, K = 16 each) and
// commits them to the chain's mbarrier, every thread of the chain waits (bounded),
// loads its row of the fp32 accumulator from the chain's 64 tensor-memory columns
// and applies the ReLU.  While one chain waits for the tensor
// cores, the other seven run their epilogues.  Weights are staged once per block,
// in the same layout, and shared by the chains.
// ---------------------------------------------------------------------------
constexpr int kRows = 128;                       // markers per tile (UMMA M) = threads per chain
constexpr int kChains = 8;                       // warpgroups per block
constexpr int kMlpThreads = kRows * kChains;     // 1024
constexpr int kTmemCols = 512;                   // chain g: columns 64 g .. 64 g + 63
constexpr int kOutN = 16;                        // output layer padded to the smallest N for M = 128

// byte offset of element (r, k) in a K-major no-swizzle operand with K columns:
// core matrix (r/8, k/8) at (r/8) * (K/8) * 128 + (k/8) * 128, row r%8 at 16 (r%8)
__host__ __device__ constexpr int kmaj_off(int r, int k, int K)
{
    return (r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

struct MlpChain {
    __nv_bfloat16 A0[kRows * 16];   // features (K = 16, 6 used)
    __nv_bfloat16 A[kRows * 64];    // hidden activations (reused per layer)
    unsigned long long bar;         // MMA completion
    int abort;
    int pad[5];
};

// The biases of layers 1-3 ride on the tensor cores: layer 1 takes b1 as weight
// column 6 against a constant feature 1; layers 2 and 3 add one K = 16 step of a
// shared block whose column 0 is 1 against a bias block whose column 0 is b.
struct MlpUmma {
    __nv_bfloat16 W1[64 * 16];      // [n][k], K = 16: 6 weights, b1, zeros
    __nv_bfloat16 W2[64 * 64];
    __nv_bfloat16 W3[64 * 64];
    __nv_bfloat16 W4[kOutN * 64];   // rows 0, 1 used
    __nv_bfloat16 ONES[kRows * 16]; // column 0 = 1
    __nv_bfloat16 B2[64 * 16];      // column 0 = b2
    __nv_bfloat16 B3[64 * 16];      // column 0 = b3
    MlpChain C[kChains];
    float b4[2];
    float norm[kNorm];
    uint32_t tmem;                  // tensor-memory base address
};

// shared-memory matrix descriptor (tcgen05): start, leading (K-direction core
// matrix) and stride (8-row group) byte offsets, version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = smem_u32(p);
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// barrier of one chain (named barrier 1 + g, its 128 threads)
__device__ __forceinline__ void chain_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kRows) : "memory");
}

// 32 consecutive fp32 columns of this thread's tensor-memory lane, and the wait
// for them, in one statement (the registers are valid only after the wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float (&v)[2])
{
    uint32_t r0, r1;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r0), "=r"(r1)
        : "r"(taddr)
        : "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
}

__device__ __forceinline__ void put_bf16(void *base, int off, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<char *>(base) + off) = __float2bfloat16(v);
}

// Stage the network (fp32 parameters in global memory) into the operand layouts.
__device__ void stage_umma(MlpUmma &S, const float *params, const float *norm)
{
    for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
        const int n = i >> 4, k = i & 15;
        put_bf16(S.W1, kmaj_off(n, k, 16),
                 k < kIn ? params[kOffW1 + n * kIn + k] : (k == kIn ? params[kOffB1 + n] : 0.f));
        put_bf16(S.B2, kmaj_off(n, k, 16), k == 0 ? params[kOffB2 + n] : 0.f);
        put_bf16(S.B3, kmaj_off(n, k, 16), k == 0 ? params[kOffB3 + n] : 0.f);
    }
    for (int i = threadIdx.x; i < kRows * 16; i += blockDim.x) {
        const int r = i >> 4, k = i & 15;
        put_bf16(S.ONES, kmaj_off(r, k, 16), k == 0 ? 1.f : 0.f);
    }
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int n = i >> 6, k = i & 63;
        put_bf16(S.W2, kmaj_off(n, k, 64), params[kOffW2 + n * kHid + k]);
        put_bf16(S.W3, kmaj_off(n, k, 64), params[kOffW3 + n * kHid + k]);
    }
    for (int i = threadIdx.x; i < kOutN * 64; i += blockDim.x) {
        const int n = i >> 6, k = i & 63;
        put_bf16(S.W4, kmaj_off(n, k, 64), n < kOut ? params[kOffW4 + n * kHid + k] : 0.f);
    }
    if (threadIdx.x < kOut) S.b4[threadIdx.x] = params[kOffB4 + threadIdx.x];
    if (threadIdx.x < kNorm) S.norm[threadIdx.x] = norm[threadIdx.x];
    // the padding half of every feature row (k = 8..15) stays zero
    const int g = threadIdx.x / kRows, r = threadIdx.x % kRows;
    *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.C[g].A0) + kmaj_off(r, 8, 16)) = make_uint4(0, 0, 0, 0);
}

// Block prologue: chain barriers, tensor memory (warp 0 allocates all 512
// columns: one block per SM), staged weights.
__device__ __forceinline__ void umma_begin(MlpUmma &S, const float *params, const float *norm)
{
    if (threadIdx.x < kChains) {
        mbar_init(&S.C[threadIdx.x].bar, 1);
        S.C[threadIdx.x].abort = 0;
    }
    if (threadIdx.x == 0) fence_mbar_init();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    stage_umma(S, params, norm);
    fence_proxy_async();           // weights and zero padding: visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void umma_end(MlpUmma &S)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(kTmemCols)
                     : "memory");
}

// Write this thread's feature row (normalised, bf16) into its chain's tile.
__device__ __forceinline__ void umma_put_features(MlpUmma &S, int g, int r, const float f[kIn])
{
    uint4 v;
    v.x = pack_bf16((f[0] - S.norm[0]) * S.norm[kIn + 0], (f[1] - S.norm[1]) * S.norm[kIn + 1]);
    v.y = pack_bf16((f[2] - S.norm[2]) * S.norm[kIn + 2], (f[3] - S.norm[3]) * S.norm[kIn + 3]);
    v.z = pack_bf16((f[4] - S.norm[4]) * S.norm[kIn + 4], (f[5] - S.norm[5]) * S.norm[kIn + 5]);
    v.w = pack_bf16(1.f, 0.f);     // feature 6 = 1 (carries b1)
    *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.C[g].A0) + kmaj_off(r, 0, 16)) = v;
}

// One layer of chain g: issue (the chain's first thread), wait (all of its
// threads); false after a bounded wait gave up.
__device__ __forceinline__ bool umma_layer(MlpUmma &S, int g, int r, const __nv_bfloat16 *Aop, int K,
                                           const __nv_bfloat16 *Bop, const __nv_bfloat16 *bias,
                                           uint32_t idesc, unsigned &phase)
{
    MlpChain &C = S.C[g];
    fence_proxy_async();           // this thread's activations: visible to the tensor cores
    tc_fence_before();
    chain_sync(g);
    tc_fence_after();
    if (r == 0) {
        const uint32_t sbo = (uint32_t)K * 16;    // K/8 core matrices of 128 bytes per 8-row group
        for (int kt = 0; kt < K / 16; ++kt)
            umma_bf16(S.tmem + 64u * g, umma_desc(reinterpret_cast<const char *>(Aop) + kt * 256, 128, sbo),
                      umma_desc(reinterpret_cast<const char *>(Bop) + kt * 256, 128, sbo), idesc, kt > 0);
        if (bias)      // + ones x bias^T
            umma_bf16(S.tmem + 64u * g, umma_desc(S.ONES, 128, 256), umma_desc(bias, 128, 256), idesc, 1u);
        umma_commit(&C.bar);
    }
    // warp 0 of the chain waits for the MMAs (bounded); the other warps block at
    // the chain barrier instead of polling
    bool ok = true;
    if (r < 32) {
        ok = mbar_wait(&C.bar, phase);
        if (!ok) atomicExch(&C.abort, 1);
        tc_fence_before();
    }
    chain_sync(g);
    if (*reinterpret_cast<volatile int *>(&C.abort)) {
        // gave up: give the MMAs in flight one more bounded wait before the block
        // frees its tensor memory and leaves
        mbar_wait(&C.bar, phase);
        ok = false;
    }
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

// ReLU of this thread's accumulator row (the chain's 64 columns, bias included)
// into its row of the next layer's operand.  Warp w reads tensor-memory lanes
// 32 (w % 4) .. + 31.
__device__ __forceinline__ void umma_epilogue(MlpUmma &S, int g, int r)
{
    const uint32_t taddr = S.tmem + ((uint32_t)(r & ~31) << 16) + 64u * g;
    char *row = reinterpret_cast<char *>(S.C[g].A);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(taddr + 32 * h, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {      // 8 columns = one 16-byte chunk of the row
            uint4 o;
            const int k0 = 32 * h + 8 * c;
            o.x = relu_bf16x2(v[8 * c + 0], v[8 * c + 1]);
            o.y = relu_bf16x2(v[8 * c + 2], v[8 * c + 3]);
            o.z = relu_bf16x2(v[8 * c + 4], v[8 * c + 5]);
            o.w = relu_bf16x2(v[8 * c + 6], v[8 * c + 7]);
            *reinterpret_cast<uint4 *>(row + kmaj_off(r, k0, 64)) = o;
        }
    }
}

// The network on chain g's 128 feature rows.  Returns false after a bounded wait
// gave up; y = this row's scaled outputs.
__device__ __forceinline__ bool umma_network(MlpUmma &S, int g, int r, unsigned &phase, float (&y)[2])
{
    constexpr uint32_t kHidDesc = idesc_bf16(kRows, kHid), kOutDesc = idesc_bf16(kRows, kOutN);
    MlpChain &C = S.C[g];
    if (!umma_layer(S, g, r, C.A0, 16, S.W1, nullptr, kHidDesc, phase)) return false;
    umma_epilogue(S, g, r);
    if (!umma_layer(S, g, r, C.A, 64, S.W2, S.B2, kHidDesc, phase)) return false;
    umma_epilogue(S, g, r);
    if (!umma_layer(S, g, r, C.A, 64, S.W3, S.B3, kHidDesc, phase)) return false;
    umma_epilogue(S, g, r);
    if (!umma_layer(S, g, r, C.A, 64, S.W4, nullptr, kOutDesc, phase)) return false;
    float o[2];
    tmem_ld2(S.tmem + ((uint32_t)(r & ~31) << 16) + 64u * g, o);
    y[0] = (o[0] + S.b4[0]) * S.norm[2 * kIn];
    y[1] = (o[1] + S.b4[1]) * S.norm[2 * kIn + 1];
    return true;
}

// ---------------------------------------------------------------------------
// Standalone inference: X (B x 6 raw features, fp32) -> Y (B x 2 scaled outputs).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMlpThreads, 1) k_mlp_infer(const float *params, const float *norm,
                                                             const float *X, long long B, float *Y, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    MlpUmma &S = *reinterpret_cast<MlpUmma *>(smem);
    umma_begin(S, params, norm);
    const int g = threadIdx.x / kRows, r = threadIdx.x % kRows;
    unsigned phase = 0;
    const long long stride = (long long)gridDim.x * kChains * kRows;
    // the next tile's inputs are loaded while the network runs on this one
    float nx[kIn];
    const long long base0 = ((long long)blockIdx.x * kChains + g) * kRows;
#pragma unroll
    for (int i = 0; i < kIn; ++i) nx[i] = base0 + r < B ? X[(base0 + r) * kIn + i] : 0.f;
    for (long long base = base0; base < B; base += stride) {
        const long long a = base + r;
        float f[kIn];
#pragma unroll
        for (int i = 0; i < kIn; ++i) f[i] = a < B ? nx[i] : S.norm[i];
        const long long an = a + stride;
#pragma unroll
        for (int i = 0; i < kIn; ++i) nx[i] = an < B ? X[an * kIn + i] : 0.f;
        umma_put_features(S, g, r, f);
        float y[2];
        if (!umma_network(S, g, r, phase, y)) {
            if (r == 0) atomicOr(status, STATUS_TIMEOUT);
            break;
        }
        if (a < B) {
            Y[2 * a] = y[0];
            Y[2 * a + 1] = y[1];
        }
    }
    umma_end(S);
}

// ---------------------------------------------------------------------------
// Warm start of subsystem I: delta^(0) = tau p/g0 + y0 dt^2/dx for every marker,
// with the features gathered at x^n from e_x^n and a^n (staged in shared memory).
// ---------------------------------------------------------------------------
template <int K, typename R>
__global__ void __launch_bounds__(kMlpThreads, 1) k_warm_mlp(WarmArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    MlpUmma &S = *reinterpret_cast<MlpUmma *>(smem);
    const int H = K + 1;
    const int W = A.M + 2 * H;
    float *s_e = reinterpret_cast<float *>(smem + ((sizeof(MlpUmma) + 127) & ~size_t(127)));
    float2 *s_a = reinterpret_cast<float2 *>(s_e + ((W + 1) & ~1));
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int gg = wrap_cell(i - H, A.M);
        s_e[i] = (float)A.ex[gg];
        s_a[i] = make_float2((float)A.ay[gg], (float)A.az[gg]);
    }
    umma_begin(S, A.params, A.norm);
    const int g = threadIdx.x / kRows, r = threadIdx.x % kRows;
    const R *tp = static_cast<const R *>(A.P.t);
    const R *pp = static_cast<const R *>(A.P.p);
    R *dp = static_cast<R *>(A.P.delta);
    const float tau = (float)(A.dt / A.dx);
    const float c2 = (float)(A.dt * A.dt / A.dx);
    unsigned phase = 0;
    const long long stride = (long long)gridDim.x * kChains * kRows;
    // the next tile's markers are loaded while the network runs on this one
    const long long base0 = ((long long)blockIdx.x * kChains + g) * kRows;
    int nc = 0;
    R nt = R(0), np_ = R(0);
    if (base0 + r < A.np) {
        nc = A.P.cell[base0 + r];
        nt = tp[base0 + r];
        np_ = pp[base0 + r];
    }
    for (long long base = base0; base < A.np; base += stride) {
        const long long a = base + r;
        const bool act = a < A.np;
        float f[kIn], pn = 0.f, g0 = 1.f;
        const int c = nc;
        const float t = (float)nt;
        pn = act ? (float)np_ : 0.f;
        if (a + stride < A.np) {
            nc = A.P.cell[a + stride];
            nt = tp[a + stride];
            np_ = pp[a + stride];
        }
        if (act) {
            float v[K + 1], u[K];
            bspline_vals<K, float>(t, v);
            bspline_vals<K - 1, float>(t, u);
            float Ay = 0.f, Az = 0.f, Ex = 0.f;
#pragma unroll
            for (int q = 0; q <= K; ++q) {
                const float2 av = s_a[c - q + H];
                Ay += av.x * v[q];
                Az += av.y * v[q];
            }
#pragma unroll
            for (int q = 0; q < K; ++q) Ex += s_e[c - q + H] * u[q];
            g0 = sqrtf(1.f + pn * pn + Ay * Ay + Az * Az);
            f[0] = t; f[1] = pn; f[2] = Ex; f[3] = Ay; f[4] = Az; f[5] = (float)A.dt;
        } else {
#pragma unroll
            for (int i = 0; i < kIn; ++i) f[i] = S.norm[i];
        }
        umma_put_features(S, g, r, f);
        float y[2];
        if (!umma_network(S, g, r, phase, y)) {
            if (r == 0) atomicOr(A.status, STATUS_TIMEOUT);
            break;
        }
        if (act) dp[a] = (R)(tau * pn / g0 + y[0] * c2);
    }
    umma_end(S);
}

// ---------------------------------------------------------------------------
// Training: loss = mean over the batch of sum_o (y_o - T_o / out_scale_o)^2 on
// the normalised outputs; gradients by the chain rule in fp32.
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
        h[s][n] = relu(acc);
    }
}

__global__ void __launch_bounds__(256) k_mlp_train(const float *params, const float *norm, const float *X,
                                                   const float *Tg, long long B, float *grad, double *loss)
{
    extern __shared__ __align__(1024) unsigned char smem[];
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
    // d3 = (dY W4) * relu'(z3)   (into d1)
    for (int i = threadIdx.x; i < ns * kHid; i += blockDim.x) {
        const int s = i / kHid, k = i % kHid;
        float acc = 0.f;
        for (int o = 0; o < kOut; ++o) acc += S.y[s][o] * S.Wt[kOffW4 + o * kHid + k];
        S.d1[s][k] = acc * relu_grad(S.z3[s][k]);
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
                dout[s][k] = acc * relu_grad(zprev[L][s][k]);
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

// Every block allocates all 512 tensor-memory columns of its SM, so only one
// block may be resident per SM (a second would wait in tcgen05.alloc): the
// shared-memory request is padded above half of the SM's.
constexpr size_t kMinUmmaSmem = 120 * 1024;

size_t mlp_infer_smem() { return sizeof(MlpUmma) > kMinUmmaSmem ? sizeof(MlpUmma) : kMinUmmaSmem; }

size_t warm_mlp_smem(int M, int K)
{
    const size_t W = (size_t)M + 2 * (size_t)(K + 1);
    const size_t s = ((sizeof(MlpUmma) + 127) & ~size_t(127)) + ((W + 1) & ~size_t(1)) * sizeof(float) +
                     W * sizeof(float2);
    return s > kMinUmmaSmem ? s : kMinUmmaSmem;
}

int launch_warm_mlp(const WarmArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = warm_mlp_smem(a.M, a.K);
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
        if (a.fp32) k_warm_mlp<KK, float><<<grid, kMlpThreads, smem, s>>>(a);                          \
        else k_warm_mlp<KK, double><<<grid, kMlpThreads, smem, s>>>(a);                                \
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
    int *status = nullptr;          // error bits of the inference kernel
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
              cudaMalloc((void **)&m->loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&m->status, sizeof(int)) == cudaSuccess;
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
    cudaFree(m->status);
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
    const size_t smem = mlp_infer_smem();
    static bool opted = false;
    if (!opted) {
        if (cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return mlp_fail(PIC_ERR_CUDA, "pic_mlp_infer: shared-memory opt-in failed");
        opted = true;
    }
    long long blocks = (B + kMlpThreads - 1) / kMlpThreads;
    if (blocks > (long long)m->num_sms) blocks = (long long)m->num_sms;
    if (cudaMemsetAsync(m->status, 0, sizeof(int), m->stream) != cudaSuccess)
        return mlp_fail(PIC_ERR_CUDA, "pic_mlp_infer: status reset failed");
    k_mlp_infer<<<(unsigned)blocks, kMlpThreads, smem, m->stream>>>(m->params, m->norm, X, B, Y, m->status);
    int st = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mlp_fail(PIC_ERR_CUDA, "pic_mlp_infer: kernel failed");
    if (st) return mlp_fail(PIC_ERR_CUDA, "pic_mlp_infer: a bounded wait on the tensor cores gave up");
    return PIC_OK;
}

// accessors for the handle code (pic_api.cu)
const float *mlp_params(const pic_mlp *m) { return m->params; }
const float *mlp_norm(const pic_mlp *m) { return m->norm; }
