// pic_noalloc.cu -- the path-integrated current deposit without any allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// deposit: code running inside a memory pool that must not grow, a host that
// has handed the whole device heap to another component, or a plugin that is
// not allowed to own CUDA allocations.  pic_deposit_current_noalloc() serves
// them: it needs no handle, and its only scratch is the file-scope device array
// below (2 MiB per GPU that loads the library, held until the process exits).
//
// Scratch layout (doubles): [0, 64) header (status word), then one row of
// W = nx + 2H partial sums per block.  Every call rewrites the rows it uses
// and clears the header first, so the contents left by the previous call do not
// leak into the result.  All calls share the array: two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race and
// corrupt each other's result; order them on one stream.
#include <cmath>
#include <mutex>

#include "pic.h"
#include "pic_internal.h"

namespace {

constexpr size_t kScratchDoubles = size_t(1) << 18;   // 2 MiB
constexpr int kHeader = 64;                            // doubles reserved for the status word
constexpr int kMaxDisp = 64;                           // cells a displacement may span
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

struct NoallocArgs {
    int M, H, nblk;
    long long np;
    double dx, w;
    const double *x, *disp;
    double *rows;       // scratch rows, nblk x W
    int *status;        // scratch header
};

// Per block: deposit its markers into a shared-memory row, then store the row.
// Inside a block the row is accumulated with shared-memory atomics, whose order
// depends on warp scheduling, so repeated calls may differ in the last bits;
// the rows of the blocks are then summed in a fixed order.
template <int K>
__global__ void __launch_bounds__(256) k_noalloc_rows(NoallocArgs A)
{
    extern __shared__ __align__(16) double s_row[];
    const int H = A.H;
    const int W = A.M + 2 * H;
    for (int i = threadIdx.x; i < W; i += blockDim.x) s_row[i] = 0.0;
    __syncthreads();
    const double wdx = A.w * A.dx;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < A.np; a += stride) {
        const double u = A.x[a] / A.dx;
        const double d = A.disp[a] / A.dx;
        // positions and displacements must be finite (an infinite position would
        // turn into NaN offsets below) and a displacement may span at most kMaxDisp cells
        if (!isfinite(u) || !isfinite(d) || !(fabs(d) <= (double)kMaxDisp)) { bad = true; continue; }
        // periodic: wrap the cell coordinate into [0, M) before taking its integer part
        const double uw = u - (double)A.M * ::floor(u / (double)A.M);
        const double f = ::floor(uw);
        double t0 = uw - f;
        int c0 = (int)f;
        if (t0 >= 1.0) { t0 = 0.0; c0 += 1; }
        c0 = pic::wrap_cell(c0, A.M);
        pic::walk_path<K, double>(t0, d, [&](int c, double h, const double *m, bool) {
            const double hw = wdx * h;
#pragma unroll
            for (int r = 0; r < K; ++r) atomicAdd(&s_row[c0 + c - r + H], hw * m[r]);
        });
    }
    if (bad) atomicOr(A.status, 1);
    __syncthreads();
    double *row = A.rows + (size_t)blockIdx.x * W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) row[i] = s_row[i];
}

// out[i] = sum over rows b (in order) of the padded entries that wrap to node i.
__global__ void __launch_bounds__(256) k_noalloc_reduce(NoallocArgs A, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.M) return;
    const int W = A.M + 2 * A.H;
    double s = 0.0;
    for (int b = 0; b < A.nblk; ++b) {
        const double *row = A.rows + (size_t)b * W;
        for (int q = i + A.H - A.M * ((i + A.H) / A.M); q < W; q += A.M) s += row[q];
    }
    out[i] = s;
}

__global__ void k_noalloc_clear(int *status) { *status = 0; }

struct DeviceSetup {
    double *scratch = nullptr;   // device address of g_scratch on this device
    int num_sms = 0;
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

// Once per device, with that device current: resolve the scratch address and
// opt the row kernels into the shared memory they need.
int setup_device(int dev, DeviceSetup **out, const char **why)
{
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSetup &d = g_dev[dev];
    if (!d.scratch) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_scratch) != cudaSuccess || !p) {
            *why = "cudaGetSymbolAddress of the deposit scratch failed";
            return PIC_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            *why = "cudaDeviceGetAttribute failed";
            return PIC_ERR_CUDA;
        }
        const int smem = (int)((8192 + 2 * (5 + kMaxDisp + 2)) * sizeof(double));
        if (cudaFuncSetAttribute(k_noalloc_rows<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ||
            cudaFuncSetAttribute(k_noalloc_rows<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ||
            cudaFuncSetAttribute(k_noalloc_rows<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ||
            cudaFuncSetAttribute(k_noalloc_rows<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) {
            *why = "cudaFuncSetAttribute failed";
            return PIC_ERR_CUDA;
        }
        d.num_sms = sms;
        d.scratch = p;
    }
    *out = &d;
    return PIC_OK;
}

int fail_nohandle(int code, const char *msg)
{
    pic::set_thread_error(msg);
    return code;
}

}  // namespace

extern "C" int pic_deposit_current_noalloc(double L, int32_t nx, int32_t degree, int64_t np,
                                           double weight, const double *x, const double *disp,
                                           double *out, void *stream)
{
    if (!(L > 0) || nx < 8 || degree < 2 || degree > 5 || np < 0 || np > 2147483647LL || !out ||
        (np > 0 && (!x || !disp)) || !std::isfinite(weight))
        return fail_nohandle(PIC_ERR_INVALID, "pic_deposit_current_noalloc: invalid argument");
    if (nx > 8192)
        return fail_nohandle(PIC_ERR_INVALID,
                             "pic_deposit_current_noalloc: nx > 8192 exceeds the fixed 2 MiB scratch");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail_nohandle(PIC_ERR_CUDA, "pic_deposit_current_noalloc: no usable current device");
    DeviceSetup *d = nullptr;
    const char *why = nullptr;
    int rc = setup_device(dev, &d, &why);
    if (rc) return fail_nohandle(rc, why);

    NoallocArgs a{};
    a.M = nx;
    a.H = degree + kMaxDisp + 2;
    const int W = a.M + 2 * a.H;
    const size_t max_rows = (kScratchDoubles - kHeader) / (size_t)W;
    a.nblk = (int)std::min<size_t>(max_rows, (size_t)d->num_sms * 2);
    if (a.nblk < 1)
        return fail_nohandle(PIC_ERR_INVALID, "pic_deposit_current_noalloc: grid too large for the scratch");
    a.np = np;
    a.dx = L / nx;
    a.w = weight;
    a.x = x;
    a.disp = disp;
    a.status = reinterpret_cast<int *>(d->scratch);
    a.rows = d->scratch + kHeader;
    k_noalloc_clear<<<1, 1, 0, s>>>(a.status);
    const size_t smem = (size_t)W * sizeof(double);
    switch (degree) {
    case 2: k_noalloc_rows<2><<<a.nblk, 256, smem, s>>>(a); break;
    case 3: k_noalloc_rows<3><<<a.nblk, 256, smem, s>>>(a); break;
    case 4: k_noalloc_rows<4><<<a.nblk, 256, smem, s>>>(a); break;
    default: k_noalloc_rows<5><<<a.nblk, 256, smem, s>>>(a); break;
    }
    k_noalloc_reduce<<<(nx + 255) / 256, 256, 0, s>>>(a, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_nohandle(PIC_ERR_CUDA, cudaGetErrorString(e));
    int status = 0;
    e = cudaMemcpyAsync(&status, a.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_nohandle(PIC_ERR_CUDA, cudaGetErrorString(e));
    if (status)
        return fail_nohandle(PIC_ERR_NUMERIC,
                             "pic_deposit_current_noalloc: a position or displacement is not finite, or a displacement spans more than 64 cells");
    return PIC_OK;
}
