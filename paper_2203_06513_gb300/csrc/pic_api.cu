// pic_api.cu -- the C ABI of libpic (declared in include/pic.h): handle,
// device memory, and the fixed-point drivers of subsystems I and II.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "pic.h"
#include "pic_handle.h"
#include "pic_internal.h"

using namespace pic;

// warm-start network accessors (pic_mlp.cu)
const float *mlp_params(const pic_mlp *m);
const float *mlp_norm(const pic_mlp *m);

int pic_set_smem_attrs(size_t s1, size_t s2, size_t s3);
static thread_local std::string g_init_error;

void pic::set_thread_error(const char *msg) { g_init_error = msg ? msg : ""; }


static const char *kVersion = "libpic 1.0 sm_103a";

static int fail(pic_handle *h, int code, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(h, PIC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// After every launch: check the launch (and, with PIC_DEBUG_SYNC=1 in the
// environment, wait for the kernel and check its completion), count it.
#define CKL_N(name)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = cudaGetLastError();                                                 \
        if (e_ == cudaSuccess && debug_sync()) e_ = cudaStreamSynchronize(h->stream);         \
        if (e_ != cudaSuccess)                                                               \
            return fail(h, PIC_ERR_CUDA, "%s (%s:%d): %s", name, __FILE__, __LINE__,          \
                        cudaGetErrorString(e_));                                             \
        ++h->launches;                                                                       \
    } while (0)
#define CKL() CKL_N("kernel")

static bool debug_sync()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("PIC_DEBUG_SYNC");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

// Device memory of the handles comes from a stream-ordered pool of the library's
// own, one per device, that keeps what destroyed handles return: a later pic_init
// in the process (the next run of a job, the runs of an ensemble) takes it back
// without mapping new memory.  Other allocators of the process are not affected.
static cudaMemPool_t handle_pool(int device)
{
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)pools.size() <= device) pools.resize(device + 1, nullptr);
    if (!pools[device]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return nullptr;
        }
        pools[device] = pool;
    }
    return pools[device];
}

template <typename T>
static int dalloc(pic_handle *h, T **p, size_t n)
{
    if (n == 0) n = 1;
    cudaMemPool_t pool = handle_pool(h->device);
    cudaError_t e = pool ? cudaMallocFromPoolAsync((void **)p, n * sizeof(T), pool, h->stream)
                         : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(h, PIC_ERR_NOMEM, "device allocation (%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    }
    return PIC_OK;
}

static void drop_graphs(pic_handle *h);

// Returns the handle's device memory to the pool (in stream order, then waits).
static void release(pic_handle *h)
{
    cudaStream_t s = h->stream;
    auto f = [s](void *p) { if (p) cudaFreeAsync(p, s); };
    for (int b = 0; b < 2; ++b) {
        f(h->Pblk[b]);
        f(h->jb[b]); f(h->sy[b]); f(h->sz[b]);
    }
    f(h->delta); f(h->pnew); f(h->a0);
    f(h->spx); f(h->spy); f(h->spz); f(h->sdy); f(h->sdz); f(h->red);
    double *arr[] = {h->ex, h->ey, h->ez, h->ay, h->az, h->ek, h->ebar, h->ga_y, h->ga_z,
                     h->eky, h->ekz, h->aky, h->akz, h->by, h->bz, h->r0y, h->r0z, h->rho,
                     h->work, h->diag, h->d_rowM0, h->d_rowM1, h->d_rowK, h->d_rowPm,
                     h->d_tapM1, h->d_tapP};
    for (double *a : arr) f(a);
    f(h->counts);
    f(h->ctrl);
    f(h->d_count);
    drop_graphs(h);
    f(h->img.a); f(h->img.f); f(h->img.an); f(h->img.ak); f(h->img.lo);
    for (int m = 0; m < kMaxStartOrder; ++m) { f(h->fh.x[m]); f(h->fh.y[m]); f(h->fh.z[m]); }
    cudaStreamSynchronize(s);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    if (h->h_count) cudaFreeHost(h->h_count);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (auto &t : h->timed) { cudaEventDestroy(t.b); cudaEventDestroy(t.e); }
    for (auto &t : h->spare) { cudaEventDestroy(t.first); cudaEventDestroy(t.second); }
    h->timed.clear();
    h->spare.clear();
}

static PartPtrs cur_parts(pic_handle *h)
{
    PartPtrs p = h->P[h->cur];
    p.delta = h->delta;
    p.pnew = h->pnew;
    return p;
}

static int sync(pic_handle *h)
{
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

static bool debug_iters()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("PIC_DEBUG_ITERS");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

static int read_ctrl(pic_handle *h)
{
    CK(cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (debug_iters()) {
        double d, e;
        memcpy(&d, &h->h_ctrl->dprev_bits, sizeof(d));
        memcpy(&e, &h->h_ctrl->eprev_bits, sizeof(e));
        fprintf(stderr, "[libpic] iter %d dmax %.3e emax %.3e status %d converged %d\n", h->h_ctrl->iter, d,
                e, h->h_ctrl->status, h->h_ctrl->converged);
    }
    return PIC_OK;
}

static int particle_grid(pic_handle *h) { return h->num_sms * 4; }

// Split runs: a sum or max over the processes that hold the plasma's markers.
static int reduce(pic_handle *h, int op, double *buf, long long n)
{
    if (!h->reduce) return PIC_OK;
    if (h->reduce(h->rctx, op, buf, (int64_t)n, (void *)h->stream) != 0)
        return fail(h, PIC_ERR_CUDA, "the split run's reduction over processes failed");
    return PIC_OK;
}

// After a sweep of a split run: the largest marker increment and the error bits of
// every process.
static int reduce_ctrl(pic_handle *h)
{
    if (!h->reduce) return PIC_OK;
    launch_split_pack(h->ctrl, h->red, h->stream);
    CKL_N("launch_split_pack");
    int rc;
    if ((rc = reduce(h, PIC_REDUCE_MAX, h->red, 3))) return rc;
    launch_split_unpack(h->ctrl, h->red, h->stream);
    CKL_N("launch_split_unpack");
    return PIC_OK;
}

static size_t a256(size_t bytes) { return (bytes + 255) & ~size_t(255); }

// Two double arrays of N_p entries in marker copy b (free between sorts): x at
// the block's start, p after it.
static void stage_doubles(pic_handle *h, int b, double **x, double **p)
{
    char *base = h->Pblk[b];
    if (x) *x = reinterpret_cast<double *>(base);
    if (p) *p = reinterpret_cast<double *>(base + a256((size_t)h->np * sizeof(double)));
}

// The device address of a page-locked host array (cudaMallocHost, cudaHostAlloc,
// cudaHostRegister), through which kernels read and write it over the host link at
// the copy engines' rate; null for pageable memory, which is staged by copies.
static const void *pinned_device_ptr(const void *hp)
{
    if (!hp) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, hp) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// degree of the time extrapolation that starts each subsystem's fixed point
constexpr int kStartOrder1 = 0;
constexpr int kStartOrder2 = 3;

// ------------------------------------------------------------------ sort
static int sort_markers(pic_handle *h)
{
    PartPtrs src = cur_parts(h);
    PartPtrs dst = h->P[1 - h->cur];
    dst.delta = h->delta;
    dst.pnew = h->pnew;
    if (launch_sort(h->fp32, h->np, h->M, h->cfg.dt / h->dx, bins_per_cell(h->np, h->M), src, dst, h->counts,
                    particle_grid(h), 256, h->stream))
        return fail(h, PIC_ERR_CUDA, "sort launch failed");
    CKL_N("launch_sort");
    h->cur = 1 - h->cur;
    return PIC_OK;
}

int pic::handle_sort(pic_handle *h) { return sort_markers(h); }
PartPtrs pic::handle_parts(pic_handle *h) { return cur_parts(h); }

pic::RunDesc pic::handle_desc(pic_handle *h)
{
    RunDesc d{};
    d.M = h->M; d.K = h->K; d.fp32 = h->fp32; d.np = h->np; d.dx = h->dx; d.dt = h->cfg.dt;
    d.P = cur_parts(h);
    d.ex = h->ex; d.ek = h->ek; d.ebar = h->ebar; d.ay = h->ay; d.az = h->az;
    d.ga_y = h->ga_y; d.ga_z = h->ga_z; d.j0 = h->jb[0]; d.j1 = h->jb[1];
    d.rowPm = h->d_rowPm; d.rowK = h->d_rowK;
    d.ey = h->ey; d.ez = h->ez; d.by = h->by; d.bz = h->bz;
    d.eky = h->eky; d.ekz = h->ekz; d.aky = h->aky; d.akz = h->akz;
    d.sy0 = h->sy[0]; d.sz0 = h->sz[0]; d.sy1 = h->sy[1]; d.sz1 = h->sz[1];
    d.ctrl = h->ctrl;
    d.img = h->img;
    d.fh = h->fh;
    return d;
}

// ------------------------------------------------------------------ charge + Poisson
static int deposit_charge(pic_handle *h, double *out)
{
    CK(cudaMemsetAsync(out, 0, sizeof(double) * h->M, h->stream));
    DiagArgs a{};
    a.M = h->M; a.K = h->K; a.fp32 = h->fp32; a.np = h->np; a.dx = h->dx; a.w = h->cfg.weight;
    a.P = cur_parts(h);
    a.out = out;
    if (launch_charge(a, particle_grid(h), 256, charge_smem(h->M, h->K + 1), h->stream))
        return fail(h, PIC_ERR_INVALID, "charge: bad degree");
    CKL_N("launch_charge");
    return PIC_OK;
}

static int conv_plain(pic_handle *h, const double *taps, int d_start, int ntap,
                      const double *in0, double *out0, const double *in1, double *out1)
{
    ConvArgs c{};
    c.M = h->M; c.d_start = d_start; c.ntap = ntap; c.mode = CONV_PLAIN; c.ncomp = in1 ? 2 : 1;
    c.taps = taps;
    c.in[0] = in0; c.in[1] = in1;
    c.out[0] = out0; c.out[1] = out1;
    c.ctrl = h->ctrl;
    if (launch_conv(c, h->stream)) return fail(h, PIC_ERR_CUDA, "k_conv shared-memory opt-in failed");
    CKL_N("launch_conv");
    return PIC_OK;
}

static int solve_poisson(pic_handle *h)
{
    int rc;
    if ((rc = deposit_charge(h, h->rho))) return rc;
    if ((rc = reduce(h, PIC_REDUCE_SUM, h->rho, h->M))) return rc;
    launch_poisson_rhs(h->M, h->dx, h->rho, h->work, h->stream);
    CKL_N("launch_poisson_rhs");
    return conv_plain(h, h->d_tapM1, h->tapM1_start, h->tapM1_n, h->work, h->ex, nullptr, nullptr);
}

// ------------------------------------------------------------------ init
extern "C" int pic_init(const pic_config *cfg, const pic_arrays *in, int32_t mem, void *stream,
                        pic_handle **out)
{
    return pic_init_split(cfg, in, mem, stream, nullptr, nullptr, out);
}

extern "C" int pic_init_split(const pic_config *cfg, const pic_arrays *in, int32_t mem, void *stream,
                              pic_reduce_fn reduce_fn, void *ctx, pic_handle **out)
{
    if (!cfg || !in || !out) return PIC_ERR_INVALID;
    *out = nullptr;
    const pic_config &c = *cfg;
    if (!(c.L > 0) || c.nx < 8 || c.nx > 8192 || c.degree < 2 || c.degree > 5 || c.np < 1 ||
        c.np > 2147483647LL || !(c.dt > 0) || !(c.tol > 0) || c.max_iter < 1 || c.max_iter > 1000 ||
        (c.precision != PIC_FP64 && c.precision != PIC_FP32) ||
        (mem != PIC_MEM_HOST && mem != PIC_MEM_DEVICE) || !in->x || !in->p || !in->ay || !in->az ||
        !std::isfinite(c.weight) || c.warm_start < 0 || c.warm_start > 2 || c.sort_every < 0 ||
        c.deposit < PIC_ACC_DEFAULT || c.deposit > PIC_ACC_DOUBLE ||
        (c.splitting != PIC_SPLIT_LIE && c.splitting != PIC_SPLIT_STRANG) || !std::isfinite(c.hbar) ||
        c.warm_field < 0 || c.warm_field > 1 || (c.warm_field && c.warm_start == PIC_WARM_NONE)) {
        g_init_error = "invalid configuration or missing input array";
        return PIC_ERR_INVALID;
    }
    if (c.hbar != 0.0 && (c.precision != PIC_FP64 || c.splitting != PIC_SPLIT_LIE ||
                          c.warm_start == PIC_WARM_MLP || !in->sx || !in->sy || !in->sz)) {
        g_init_error = "spin (hbar != 0) needs the FP64 form, Lie--Trotter steps, no learned warm start "
                       "and the sx, sy, sz arrays";
        return PIC_ERR_INVALID;
    }
    const double dx = c.L / c.nx;
    if (c.dt / dx > 64.0) {
        g_init_error = "dt/dx > 64";
        return PIC_ERR_INVALID;
    }

    pic_handle *h = new (std::nothrow) pic_handle();
    if (!h) return PIC_ERR_NOMEM;
    h->cfg = c;
    h->stream = (cudaStream_t)stream;
    h->reduce = reduce_fn;
    h->rctx = ctx;
    h->M = c.nx;
    h->K = c.degree;
    h->np = c.np;
    h->dx = dx;
    h->fp32 = c.precision == PIC_FP32;
    h->rsize = h->fp32 ? sizeof(float) : sizeof(double);
    if (!h->fp32) {
        h->acc = ACC_NATIVE;                    // double lanes: the FP64 form
        if (c.deposit != PIC_ACC_DEFAULT && c.deposit != PIC_ACC_DOUBLE) {
            g_init_error = "the FP64 form accumulates deposits in double (deposit must be default or double)";
            delete h;
            return PIC_ERR_INVALID;
        }
    } else {
        h->acc = c.deposit == PIC_ACC_FLOAT ? ACC_NATIVE : c.deposit == PIC_ACC_DOUBLE ? ACC_DOUBLE : ACC_COMP;
    }
    if (!sweep_variant_ok(c.degree, h->fp32, h->acc)) {
        g_init_error = "this deposit accumulation is built for degrees 3 and 5 only";
        delete h;
        return PIC_ERR_INVALID;
    }
    // |x^{n+1} - x^n| < dt because |p|/gamma < 1: at most ceil(dt/dx) cells
    h->Dlim = (int)std::ceil(c.dt / dx) + 1;
    h->H = h->K + h->Dlim + 2;
    int rc = PIC_OK;
    auto bail = [&](int code) {
        g_init_error = h->err.empty() ? "pic_init failed" : h->err;
        release(h);
        delete h;
        return code;
    };

    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(PIC_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return bail(PIC_ERR_CUDA);

    const size_t np = (size_t)h->np, M = (size_t)h->M;
    // marker arrays are padded by 64 entries: the sweeps' bulk copies round a
    // tile's byte count up to a multiple of 16 and may read up to 3 entries past N_p
    const size_t npa = np + 64;
    // each copy: cell, t, p, id back to back, every array 256-byte aligned; at least
    // 16 bytes a marker, room for the staged (x, p) doubles of a host transfer
    const size_t off_t = a256(npa * sizeof(int32_t)), off_p = off_t + a256(npa * h->rsize);
    const size_t off_id = off_p + a256(npa * h->rsize), blk = off_id + a256(npa * sizeof(int32_t));
    for (int b = 0; b < 2; ++b) {
        if ((rc = dalloc(h, &h->Pblk[b], blk))) return bail(rc);
        h->P[b].cell = reinterpret_cast<int32_t *>(h->Pblk[b]);
        h->P[b].t = h->Pblk[b] + off_t;
        h->P[b].p = h->Pblk[b] + off_p;
        h->P[b].id = reinterpret_cast<int32_t *>(h->Pblk[b] + off_id);
        if ((rc = dalloc(h, &h->jb[b], M))) return bail(rc);
        if ((rc = dalloc(h, &h->sy[b], M))) return bail(rc);
        if ((rc = dalloc(h, &h->sz[b], M))) return bail(rc);
    }
    if ((rc = dalloc(h, (char **)&h->delta, npa * h->rsize))) return bail(rc);
    if ((rc = dalloc(h, (char **)&h->pnew, npa * h->rsize))) return bail(rc);
    // the start-point cache pays in the FP64 form (its arithmetic runs on the narrow
    // FP64 pipe: 311 -> 287 ms a step on C2); in the FP32 form the extra 16 bytes a
    // marker cost more than the instructions they save (1.98 -> 2.04 ms a sweep)
    if (!h->fp32 && (rc = dalloc(h, (char **)&h->a0, npa * 4 * h->rsize))) return bail(rc);
    double **grid_arrays[] = {&h->ex, &h->ey, &h->ez, &h->ay, &h->az, &h->ek, &h->ebar, &h->ga_y,
                              &h->ga_z, &h->eky, &h->ekz, &h->aky, &h->akz, &h->by, &h->bz,
                              &h->r0y, &h->r0z, &h->rho, &h->work};
    for (double **a : grid_arrays)
        if ((rc = dalloc(h, a, M))) return bail(rc);
    // starting fields: subsystem I from e_x^n (its changes are dominated by marker
    // noise, which no extrapolation predicts); subsystem II cubic in time (the
    // transverse fields are smooth waves)
    h->fh.order1 = kStartOrder1;
    h->fh.order2 = kStartOrder2;
    for (int m = 0; m < kMaxStartOrder; ++m) {
        double **arr[] = {&h->fh.x[m], &h->fh.y[m], &h->fh.z[m]};
        const int order[] = {h->fh.order1, h->fh.order2, h->fh.order2};
        for (int c = 0; c < 3; ++c) {
            if (m >= order[c]) continue;
            if ((rc = dalloc(h, arr[c], M))) return bail(rc);
            if (cudaMemsetAsync(*arr[c], 0, sizeof(double) * M, h->stream) != cudaSuccess) return bail(PIC_ERR_CUDA);
        }
    }
    if ((rc = dalloc(h, &h->diag, 8))) return bail(rc);
    if (reduce_fn && (rc = dalloc(h, &h->red, 4))) return bail(rc);
    if (c.hbar != 0.0) {
        if ((rc = dalloc(h, &h->spx, np)) || (rc = dalloc(h, &h->spy, np)) || (rc = dalloc(h, &h->spz, np)) ||
            (rc = dalloc(h, &h->sdy, M)) || (rc = dalloc(h, &h->sdz, M)))
            return bail(rc);
        const cudaMemcpyKind k = mem == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        cudaMemcpyAsync(h->spx, in->sx, np * sizeof(double), k, h->stream);
        cudaMemcpyAsync(h->spy, in->sy, np * sizeof(double), k, h->stream);
        cudaMemcpyAsync(h->spz, in->sz, np * sizeof(double), k, h->stream);
        if (spin_optin(h->M)) return bail(fail(h, PIC_ERR_CUDA, "spin deposit shared-memory opt-in failed"));
    }
    if (h->fp32) {
        if ((rc = dalloc(h, &h->img.a, M)) || (rc = dalloc(h, &h->img.f, M)) || (rc = dalloc(h, &h->img.an, M)) ||
            (rc = dalloc(h, &h->img.ak, M)) || (rc = dalloc(h, &h->img.lo, M)))
            return bail(rc);
        double fact = 1.0;
        for (int d = 2; d <= c.degree; ++d) fact *= d;
        h->img.inv_fact = 1.0 / fact;
        h->img.escale = dx / (double)mean_scale(c.degree - 1);
    }
    if ((rc = dalloc(h, &h->counts, 2 * M * kVelBinsBase * bins_per_cell((long long)np, (int)M)))) return bail(rc);
    if ((rc = dalloc(h, &h->ctrl, 1))) return bail(rc);
    if (cudaMallocHost((void **)&h->h_flag, sizeof(int)) != cudaSuccess) return bail(PIC_ERR_NOMEM);
    if (cudaMallocHost((void **)&h->h_ctrl, sizeof(DevCtrl)) != cudaSuccess) return bail(PIC_ERR_NOMEM);

    // circulant bands: M0 (degree k), M1 (degree k-1), K = G^T M1 G, P = M0 +/- dt^2/4 K
    const int K = h->K;
    std::vector<double> m0(K + 1, 0.0), m1(K + 1, 0.0), kr(K + 1, 0.0), pp(K + 1), pm(K + 1);
    mass_band(K, dx, m0.data());
    mass_band(K - 1, dx, m1.data());
    // K_d = (2 m1_d - m1_{d-1} - m1_{d+1}) / dx^2 with m1_{-d} = m1_d
    auto m1at = [&](int d) { d = std::abs(d); return d <= K - 1 ? m1[d] : 0.0; };
    for (int d = 0; d <= K; ++d) kr[d] = (2.0 * m1at(d) - m1at(d - 1) - m1at(d + 1)) / (dx * dx);
    const double q = c.dt * c.dt / 4.0;
    for (int d = 0; d <= K; ++d) { pp[d] = m0[d] + q * kr[d]; pm[d] = m0[d] - q * kr[d]; }
    std::vector<double> gfull(M), taps(M);
    if ((rc = dalloc(h, &h->d_rowM0, K + 1))) return bail(rc);
    if ((rc = dalloc(h, &h->d_rowM1, K + 1))) return bail(rc);
    if ((rc = dalloc(h, &h->d_rowK, K + 1))) return bail(rc);
    if ((rc = dalloc(h, &h->d_rowPm, K + 1))) return bail(rc);
    cudaMemcpyAsync(h->d_rowM0, m0.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->d_rowM1, m1.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->d_rowK, kr.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->d_rowPm, pm.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, h->stream);
    {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return bail(fail(h, PIC_ERR_CUDA, "band upload: %s", cudaGetErrorString(e)));
    }
    // truncate the inverse rows where they fall below 1e-17 of their largest entry:
    // above the rounding noise of the double DFT that forms them (about 1e-18), and
    // the dropped geometric tail changes a solve by far less than one double ulp
    const double cut = 1e-17;
    inverse_taps(m1.data(), K - 1, h->M, cut, gfull.data(), &h->tapM1_start, &h->tapM1_n, taps.data());
    if ((rc = dalloc(h, &h->d_tapM1, h->tapM1_n))) return bail(rc);
    if (cudaMemcpy(h->d_tapM1, taps.data(), sizeof(double) * h->tapM1_n, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(PIC_ERR_CUDA);
    inverse_taps(pp.data(), K, h->M, cut, gfull.data(), &h->tapP_start, &h->tapP_n, taps.data());
    if ((rc = dalloc(h, &h->d_tapP, h->tapP_n))) return bail(rc);
    if (cudaMemcpy(h->d_tapP, taps.data(), sizeof(double) * h->tapP_n, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(PIC_ERR_CUDA);

    // shared-memory budgets and persistent grid size
    h->smem1 = sweep1_smem(h->M, h->H, h->fp32);
    h->smem2 = sweep2_smem(h->M, h->H, h->fp32);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (h->smem1 > (size_t)maxsm || h->smem2 > (size_t)maxsm) {
        fail(h, PIC_ERR_INVALID, "grid too large for shared memory (%zu > %d)", h->smem1, maxsm);
        return bail(PIC_ERR_INVALID);
    }
    // opt in to large dynamic shared memory (per kernel instantiation), then size the
    // persistent sweep grids as SMs x resident blocks per SM
    if (pic_set_smem_attrs(std::max(h->smem1, h->smem2), std::max(h->smem1, h->smem2),
                           charge_smem(h->M, h->H)))
        return bail(fail(h, PIC_ERR_CUDA, "cudaFuncSetAttribute failed"));
    {
        const int b1 = sweep_blocks_per_sm(h->K, h->fp32, h->acc, 1, h->sweep_block, h->smem1);
        const int b2 = sweep_blocks_per_sm(h->K, h->fp32, h->acc, 2, h->sweep_block, h->smem2);
        if (b1 < 1 || b2 < 1) return bail(fail(h, PIC_ERR_INVALID, "sweep kernels do not fit on an SM"));
        h->sweep_grid = h->num_sms * std::min(b1, b2);
    }

    // inputs
    {
        const double *dx_in = in->x, *dp_in = in->p;
        const bool host = mem == PIC_MEM_HOST;
        if (host) {
            // page-locked host arrays are read by the load kernel itself; others are
            // staged in the second marker copy, which the first sort overwrites
            const double *px = static_cast<const double *>(pinned_device_ptr(in->x));
            const double *pp = static_cast<const double *>(pinned_device_ptr(in->p));
            double *sx = nullptr, *sp = nullptr;
            stage_doubles(h, 1, &sx, &sp);
            if (px) dx_in = px;
            else { cudaMemcpyAsync(sx, in->x, np * sizeof(double), cudaMemcpyHostToDevice, h->stream); dx_in = sx; }
            if (pp) dp_in = pp;
            else { cudaMemcpyAsync(sp, in->p, np * sizeof(double), cudaMemcpyHostToDevice, h->stream); dp_in = sp; }
        }
        const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        cudaMemcpyAsync(h->ay, in->ay, M * sizeof(double), kind, h->stream);
        cudaMemcpyAsync(h->az, in->az, M * sizeof(double), kind, h->stream);
        if (in->ey) cudaMemcpyAsync(h->ey, in->ey, M * sizeof(double), kind, h->stream);
        else cudaMemsetAsync(h->ey, 0, M * sizeof(double), h->stream);
        if (in->ez) cudaMemcpyAsync(h->ez, in->ez, M * sizeof(double), kind, h->stream);
        else cudaMemsetAsync(h->ez, 0, M * sizeof(double), h->stream);
        PartPtrs P0 = h->P[0];
        P0.delta = h->delta;
        P0.pnew = h->pnew;
        launch_load(h->fp32, h->np, h->M, dx, dx_in, dp_in, P0, particle_grid(h), 256, h->stream);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return bail(fail(h, PIC_ERR_CUDA, "input copies / load: %s", cudaGetErrorString(e)));
    }
    if (launch_ctrl_reset(h->ctrl, h->stream) || cudaGetLastError() != cudaSuccess) return bail(PIC_ERR_CUDA);
    h->cur = 0;
    if ((rc = sort_markers(h))) return bail(rc);
    if ((rc = solve_poisson(h))) return bail(rc);
    if ((rc = sync(h))) return bail(rc);
    *out = h;
    return PIC_OK;
}

// ------------------------------------------------------------------ substeps
static int check_status(pic_handle *h, int which)
{
    if (h->h_ctrl->status & STATUS_TIMEOUT)
        return fail(h, PIC_ERR_CUDA, "subsystem %d: a bounded wait on a bulk copy gave up", which);
    if (h->h_ctrl->status & STATUS_NUMERIC)
        return fail(h, PIC_ERR_NUMERIC, "subsystem %d: non-finite value or displacement beyond c dt", which);
    if (h->h_ctrl->status & STATUS_NOCONV)
        return fail(h, PIC_ERR_NOCONVERGE, "subsystem %d: no convergence in %d sweeps", which,
                    h->cfg.max_iter);
    return PIC_OK;
}

// Timing without host synchronisation: each timed launch gets its own pair of
// events, recorded on the handle's stream; the pairs are read when the timing
// is read (or when many are pending) and then reused.
constexpr size_t kMaxTimedLaunches = 4096;
static int timing_fold(pic_handle *h);

static int timed_begin(pic_handle *h)
{
    if (!h->timing) return PIC_OK;
    int rc;
    if (h->timed.size() >= kMaxTimedLaunches && (rc = timing_fold(h))) return rc;
    if (h->spare.empty()) {
        cudaEvent_t b = nullptr, e = nullptr;
        CK(cudaEventCreate(&b));
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaEventDestroy(b);
            return fail(h, PIC_ERR_CUDA, "cudaEventCreate failed");
        }
        h->spare.emplace_back(b, e);
    }
    CK(cudaEventRecord(h->spare.back().first, h->stream));
    return PIC_OK;
}

static int timed_end(pic_handle *h, int kind)
{
    if (!h->timing) return PIC_OK;
    auto pr = h->spare.back();
    h->spare.pop_back();
    h->timed.push_back({pr.first, pr.second, kind});
    CK(cudaEventRecord(pr.second, h->stream));
    return PIC_OK;
}

// Adds the pending pairs' durations to the totals and returns the pairs to the spares.
static int timing_fold(pic_handle *h)
{
    if (h->timed.empty()) return PIC_OK;
    CK(cudaEventSynchronize(h->timed.back().e));
    for (auto &t : h->timed) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t.b, t.e));
        double *acc[] = {&h->t_sw1, &h->t_sw2, &h->t_solve, &h->t_warm};
        long long *cnt[] = {&h->n_sw1, &h->n_sw2, &h->n_solve, &h->n_warm};
        *acc[t.kind] += ms;
        ++*cnt[t.kind];
        h->spare.emplace_back(t.b, t.e);
    }
    h->timed.clear();
    return PIC_OK;
}

static SpinArgs spin_args(pic_handle *h)
{
    SpinArgs a{};
    a.M = h->M; a.K = h->K; a.np = h->np; a.dx = h->dx; a.w = h->cfg.weight; a.dt = h->cfg.dt;
    a.hbar = h->cfg.hbar;
    a.P = cur_parts(h);
    a.ay = h->ay; a.az = h->az;
    a.sx = h->spx; a.sy = h->spy; a.sz = h->spz;
    a.dy = h->sdy; a.dz = h->sdz;
    a.acc = h->diag + 6;
    return a;
}

// Subsystem III: the exact rotation of every spin (markers and fields frozen).
static int substep3(pic_handle *h)
{
    if (h->cfg.hbar == 0.0) return fail(h, PIC_ERR_INVALID, "subsystem III needs hbar != 0");
    if (launch_spin_rotate(spin_args(h), particle_grid(h), h->stream)) return fail(h, PIC_ERR_INVALID, "bad degree");
    CKL_N("launch_spin_rotate");
    return PIC_OK;
}

// Subsystem I over a time step dt (the handle's dt, or half of it in a Strang step).
static Sweep1Args sweep1_args(pic_handle *h, double dt)
{
    Sweep1Args a{};
    a.M = h->M; a.H = h->H; a.Dlim = h->Dlim; a.K = h->K; a.fp32 = h->fp32; a.acc = h->acc; a.np = h->np;
    a.dx = h->dx; a.dt = dt; a.w = h->cfg.weight;
    a.P = cur_parts(h);
    a.ebar = h->ebar; a.ga_y = h->ga_y; a.ga_z = h->ga_z; a.ay = h->ay; a.az = h->az;
    a.ctrl = h->ctrl;
    a.img = h->img;
    a.a0 = h->a0;
    a.hbar = h->cfg.hbar;
    a.sy = h->spy;
    a.sz = h->spz;
    a.jpair[0] = h->jb[0]; a.jpair[1] = h->jb[1];
    return a;
}

static ConvArgs conv1_args(pic_handle *h, double dt)
{
    ConvArgs c{};
    c.img = h->img;
    c.M = h->M; c.d_start = h->tapM1_start; c.ntap = h->tapM1_n; c.mode = CONV_SOLVE1; c.ncomp = 1;
    c.taps = h->d_tapM1;
    c.en[0] = h->ex; c.ek[0] = h->ek; c.aux[0] = h->ebar;
    c.dt = dt; c.dx = h->dx; c.tol = h->cfg.tol; c.dtol = 1e-6;   // FP32: estimated position error, cells relative to max(1, |delta|)
    c.erel = h->cfg.warm_field ? kFieldIncrementRelPredicted : kFieldIncrementRel;
    c.max_iter = h->cfg.max_iter; c.fp32 = h->fp32; c.subsystem = 1; c.ctrl = h->ctrl;
    c.pair[0][0] = h->jb[0]; c.pair[0][1] = h->jb[1];
    return c;
}

static Sweep2Args sweep2_args(pic_handle *h)
{
    Sweep2Args a{};
    a.status = &h->ctrl->status;
    a.M = h->M; a.H = h->H; a.K = h->K; a.fp32 = h->fp32; a.acc = h->acc; a.np = h->np; a.w = h->cfg.weight;
    a.P = cur_parts(h);
    a.an_y = h->ay; a.an_z = h->az; a.ak_y = h->aky; a.ak_z = h->akz;
    a.img = h->img;
    a.ctrl = h->ctrl;
    a.sypair[0] = h->sy[0]; a.sypair[1] = h->sy[1];
    a.szpair[0] = h->sz[0]; a.szpair[1] = h->sz[1];
    return a;
}

static ConvArgs conv2_args(pic_handle *h)
{
    ConvArgs c{};
    c.img = h->img;
    c.M = h->M; c.d_start = h->tapP_start; c.ntap = h->tapP_n; c.mode = CONV_SOLVE2; c.ncomp = 2;
    c.taps = h->d_tapP;
    c.en[0] = h->ey; c.en[1] = h->ez; c.ek[0] = h->eky; c.ek[1] = h->ekz;
    c.aux[0] = h->aky; c.aux[1] = h->akz; c.an[0] = h->ay; c.an[1] = h->az;
    c.r0[0] = h->r0y; c.r0[1] = h->r0z;
    c.dt = h->cfg.dt; c.dx = h->dx; c.tol = h->cfg.tol; c.dtol = 0.0;
    c.max_iter = h->cfg.max_iter; c.fp32 = h->fp32; c.subsystem = 2; c.ctrl = h->ctrl;
    c.pair[0][0] = h->sy[0]; c.pair[0][1] = h->sy[1];
    c.pair[1][0] = h->sz[0]; c.pair[1][1] = h->sz[1];
    return c;
}

static WarmArgs warm_args(pic_handle *h, double dt)
{
    WarmArgs wa{};
    wa.M = h->M; wa.K = h->K; wa.fp32 = h->fp32; wa.np = h->np; wa.dx = h->dx; wa.dt = dt;
    wa.P = cur_parts(h);
    wa.ex = h->ex; wa.ay = h->ay; wa.az = h->az;
    wa.params = mlp_params(h->mlp); wa.norm = mlp_norm(h->mlp);
    wa.status = &h->ctrl->status;
    return wa;
}

// The predicted start of subsystem I (warm_field): delta^(0) and j^(0) into jb[1]
// (cleared by the preparation; the first sweep deposits into jb[0] and its solve
// clears jb[1]), then e^(0) = e^n - M1^{-1} j^(0) and ebar^(0).
static int predicted_start(pic_handle *h, double dt, cudaStream_t s)
{
    Sweep1Args a = sweep1_args(h, dt);
    a.warm = h->cfg.warm_start == PIC_WARM_EXPLICIT ? 1 : 0;   // else the network's delta is there
    a.j = h->jb[1];
    a.first = 1;
    if (launch_predeposit(a, h->sweep_grid, h->sweep_block, h->smem1, s))
        return fail(h, PIC_ERR_INVALID, "predeposit");
    int rc;
    if (s == h->stream && (rc = reduce(h, PIC_REDUCE_SUM, h->jb[1], h->M))) return rc;   // split runs
    ConvArgs c = conv1_args(h, dt);
    c.mode = CONV_START1;
    c.in[0] = h->jb[1];
    if (launch_conv(c, s)) return fail(h, PIC_ERR_CUDA, "k_conv launch");
    return PIC_OK;
}

static int substep1(pic_handle *h, int *iters, double dt)
{
    int rc;
    const RunDesc desc = handle_desc(h);
    launch_prep1(desc, h->stream);
    CKL_N("launch_prep1");
    Sweep1Args a = sweep1_args(h, dt);
    ConvArgs c = conv1_args(h, dt);
    if (h->cfg.warm_start == PIC_WARM_MLP) {
        // learned proposal for delta^(0), written over the zero iterate
        if (!h->mlp) return fail(h, PIC_ERR_INVALID, "warm_start = PIC_WARM_MLP but no network attached");
        const WarmArgs wa = warm_args(h, dt);
        if ((rc = timed_begin(h))) return rc;
        if (launch_warm_mlp(wa, h->num_sms, h->stream))
            return fail(h, PIC_ERR_CUDA, "warm-start network: launch setup failed");
        CKL_N("launch_warm_mlp");
        if ((rc = timed_end(h, 3))) return rc;
    }
    if (h->cfg.warm_field) {
        if ((rc = predicted_start(h, dt, h->stream))) return rc;
        CKL_N("predicted start");
        ++h->launches;
    }
    int it = 0;
    for (;;) {
        a.j = h->jb[it & 1];
        a.warm = (it == 0 && h->cfg.warm_start == PIC_WARM_EXPLICIT && !h->cfg.warm_field) ? 1 : 0;
        a.first = it == 0 ? 1 : 0;
        if ((rc = timed_begin(h))) return rc;
        if (launch_sweep1(a, h->sweep_grid, h->sweep_block, h->smem1, h->stream))
            return fail(h, PIC_ERR_INVALID, "sweep1: bad degree");
        CKL_N("launch_sweep1");
        if ((rc = timed_end(h, 0))) return rc;
        h->marker_sweeps += h->np;
        if ((rc = reduce(h, PIC_REDUCE_SUM, h->jb[it & 1], h->M)) || (rc = reduce_ctrl(h))) return rc;
        c.in[0] = h->jb[it & 1];
        c.zero[0] = h->jb[(it + 1) & 1];
        if ((rc = timed_begin(h))) return rc;
        if (launch_conv(c, h->stream)) return fail(h, PIC_ERR_CUDA, "k_conv shared-memory opt-in failed");
        CKL_N("launch_conv");
        if ((rc = timed_end(h, 2))) return rc;
        ++it;
        if ((rc = read_ctrl(h))) return rc;
        if (h->h_ctrl->converged) break;
    }
    if (iters) *iters = it;
    if ((rc = check_status(h, 1))) return rc;
    launch_finalize1(h->fp32, h->np, h->M, cur_parts(h), h->cfg.warm_start == PIC_WARM_NONE, particle_grid(h), 256,
                     h->stream);
    CKL_N("launch_finalize1");
    launch_commit(desc, 1, h->stream);
    CKL_N("launch_commit");
    return PIC_OK;
}

static int substep2(pic_handle *h, int *iters)
{
    int rc;
    const RunDesc desc = handle_desc(h);
    launch_prep2(desc, h->stream);
    CKL_N("launch_prep2");
    if (h->cfg.hbar != 0.0) {
        // Zeeman source of the right side (constant during the loop: x, s frozen)
        SpinArgs sa = spin_args(h);
        CK(cudaMemsetAsync(h->sdy, 0, sizeof(double) * h->M, h->stream));
        CK(cudaMemsetAsync(h->sdz, 0, sizeof(double) * h->M, h->stream));
        if (launch_spin_deposit(sa, particle_grid(h), h->stream)) return fail(h, PIC_ERR_INVALID, "bad degree");
        CKL_N("launch_spin_deposit");
        if ((rc = reduce(h, PIC_REDUCE_SUM, h->sdy, h->M)) || (rc = reduce(h, PIC_REDUCE_SUM, h->sdz, h->M)))
            return rc;
        launch_spin_rhs(h->M, h->dx, h->cfg.dt, h->cfg.hbar, h->sdy, h->sdz, h->by, h->bz, h->stream);
        CKL_N("launch_spin_rhs");
    }
    if ((rc = conv_plain(h, h->d_tapP, h->tapP_start, h->tapP_n, h->by, h->r0y, h->bz, h->r0z))) return rc;
    Sweep2Args a = sweep2_args(h);
    ConvArgs c = conv2_args(h);
    int it = 0;
    for (;;) {
        a.s_y = h->sy[it & 1];
        a.s_z = h->sz[it & 1];
        if ((rc = timed_begin(h))) return rc;
        if (launch_sweep2(a, h->sweep_grid, h->sweep_block, h->smem2, h->stream))
            return fail(h, PIC_ERR_INVALID, "sweep2: bad degree");
        CKL_N("launch_sweep2");
        if ((rc = timed_end(h, 1))) return rc;
        if ((rc = reduce(h, PIC_REDUCE_SUM, h->sy[it & 1], h->M)) ||
            (rc = reduce(h, PIC_REDUCE_SUM, h->sz[it & 1], h->M)) || (rc = reduce_ctrl(h)))
            return rc;
        c.in[0] = h->sy[it & 1];
        c.in[1] = h->sz[it & 1];
        c.zero[0] = h->sy[(it + 1) & 1];
        c.zero[1] = h->sz[(it + 1) & 1];
        if ((rc = timed_begin(h))) return rc;
        if (launch_conv(c, h->stream)) return fail(h, PIC_ERR_CUDA, "k_conv shared-memory opt-in failed");
        CKL_N("launch_conv");
        if ((rc = timed_end(h, 2))) return rc;
        ++it;
        if ((rc = read_ctrl(h))) return rc;
        if (h->h_ctrl->converged) break;
    }
    if (iters) *iters = it;
    if ((rc = check_status(h, 2))) return rc;
    // a^{n+1} = a^n - dt/2 (e^n + e^{n+1}) is the last a^(k); e^{n+1} the last e^(k)
    launch_commit(desc, 2, h->stream);
    CKL_N("launch_commit");
    return PIC_OK;
}

extern "C" int pic_substep(pic_handle *h, int32_t which, int32_t *iters)
{
    if (!h) return PIC_ERR_INVALID;
    int it = 0, rc;
    if (which == PIC_SUBSYSTEM_I) rc = substep1(h, &it, h->cfg.dt);
    else if (which == PIC_SUBSYSTEM_II) rc = substep2(h, &it);
    else if (which == PIC_SUBSYSTEM_III) rc = substep3(h);
    else return fail(h, PIC_ERR_INVALID, "which must be 1, 2 or 3");
    if (iters) *iters = it;
    if (rc) return rc;
    return sync(h);
}

// ------------------------------------------------------------------ step graphs
// One step as a CUDA graph: the linear segments as child graphs, the two
// fixed-point loops as conditional WHILE nodes whose bodies (sweep, solve) read
// the sweep's parity from the control block and whose solve takes the loop's
// decision on the device (no host round trip per sweep).  The markers' buffers
// enter the kernel arguments, so there is one graph per marker copy (the sort
// alternates them).  Host loops are kept for split runs (their reductions call
// back into the host), spin runs, kernel timing and PIC_DEBUG_SYNC.
static bool graph_eligible(const pic_handle *h)
{
    return !h->reduce && h->cfg.hbar == 0.0 && !h->timing && !debug_sync() &&
           (h->cfg.warm_start != PIC_WARM_MLP || h->mlp) && getenv("PIC_NO_GRAPH") == nullptr;
}

static void drop_graphs(pic_handle *h)
{
    for (int b = 0; b < 2; ++b)
        if (h->step_exec[b]) {
            cudaGraphExecDestroy(h->step_exec[b]);
            h->step_exec[b] = nullptr;
        }
}

#define GCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(h, PIC_ERR_CUDA, "step graph: %s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static int seg_sub1_head(pic_handle *h, cudaStream_t s, double dt, int *nodes)
{
    launch_prep1(handle_desc(h), s);
    ++*nodes;
    if (h->cfg.warm_start == PIC_WARM_MLP) {
        if (launch_warm_mlp(warm_args(h, dt), h->num_sms, s)) return fail(h, PIC_ERR_CUDA, "warm-start launch");
        ++*nodes;
    }
    if (h->cfg.warm_field) {
        int rc;
        if ((rc = predicted_start(h, dt, s))) return rc;
        *nodes += 2;
    }
    return PIC_OK;
}

static int seg_sub1_tail(pic_handle *h, cudaStream_t s, int *nodes)
{
    launch_finalize1(h->fp32, h->np, h->M, cur_parts(h), h->cfg.warm_start == PIC_WARM_NONE, particle_grid(h), 256,
                     s);
    launch_commit(handle_desc(h), 1, s);
    *nodes += 2;
    return PIC_OK;
}

static int seg_sub2_head(pic_handle *h, cudaStream_t s, int *nodes)
{
    launch_prep2(handle_desc(h), s);
    ConvArgs c{};
    c.M = h->M; c.d_start = h->tapP_start; c.ntap = h->tapP_n; c.mode = CONV_PLAIN; c.ncomp = 2;
    c.taps = h->d_tapP;
    c.in[0] = h->by; c.in[1] = h->bz;
    c.out[0] = h->r0y; c.out[1] = h->r0z;
    c.ctrl = h->ctrl;
    if (launch_conv(c, s)) return fail(h, PIC_ERR_CUDA, "k_conv launch");
    *nodes += 2;
    return PIC_OK;
}

static int seg_sub2_tail(pic_handle *h, cudaStream_t s, int *nodes)
{
    launch_commit(handle_desc(h), 2, s);
    *nodes += 1;
    return PIC_OK;
}

static int loop_body(pic_handle *h, cudaStream_t s, int which, double dt, unsigned long long cond)
{
    if (which == 1) {
        Sweep1Args a = sweep1_args(h, dt);
        a.graph = 1;
        a.warm = (h->cfg.warm_start == PIC_WARM_EXPLICIT && !h->cfg.warm_field) ? 1 : 0;   // applied when iter == 0
        a.j = h->jb[0];
        if (launch_sweep1(a, h->sweep_grid, h->sweep_block, h->smem1, s)) return fail(h, PIC_ERR_INVALID, "sweep1");
        ConvArgs c = conv1_args(h, dt);
        c.graph = 1;
        c.cond_handle = cond;
        c.count = h->d_count;
        if (launch_conv(c, s)) return fail(h, PIC_ERR_CUDA, "k_conv launch");
    } else {
        Sweep2Args a = sweep2_args(h);
        a.graph = 1;
        a.s_y = h->sy[0];
        a.s_z = h->sz[0];
        if (launch_sweep2(a, h->sweep_grid, h->sweep_block, h->smem2, s)) return fail(h, PIC_ERR_INVALID, "sweep2");
        ConvArgs c = conv2_args(h);
        c.graph = 1;
        c.cond_handle = cond;
        c.count = h->d_count + 1;
        if (launch_conv(c, s)) return fail(h, PIC_ERR_CUDA, "k_conv launch");
    }
    return PIC_OK;
}

static int build_step_graph(pic_handle *h)
{
    if (!h->cap) GCK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    GCK(cudaGraphCreate(&g, 0));
    cudaGraphNode_t prev = nullptr;
    int nodes = 0;
    auto add_segment = [&](auto &&seg) -> int {
        cudaGraph_t child = nullptr;
        GCK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        const int r = seg(h->cap);
        cudaError_t ce = cudaStreamEndCapture(h->cap, &child);
        if (r) { if (child) cudaGraphDestroy(child); return r; }
        GCK(ce);
        cudaGraphNode_t n = nullptr;
        ce = cudaGraphAddChildGraphNode(&n, g, prev ? &prev : nullptr, prev ? 1 : 0, child);
        cudaGraphDestroy(child);
        GCK(ce);
        prev = n;
        return PIC_OK;
    };
    auto add_loop = [&](int which, double dt) -> int {
        cudaGraphConditionalHandle hnd;
        GCK(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = hnd;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t n = nullptr;
        GCK(cudaGraphAddNode(&n, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        GCK(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const int r = loop_body(h, h->cap, which, dt, (unsigned long long)hnd);
        cudaError_t ce = cudaStreamEndCapture(h->cap, &body);
        if (r) return r;
        GCK(ce);
        prev = n;
        return PIC_OK;
    };
    const bool strang = h->cfg.splitting == PIC_SPLIT_STRANG;
    const double dt1 = strang ? 0.5 * h->cfg.dt : h->cfg.dt;
    int rc = PIC_OK;
    if (!rc) rc = add_segment([&](cudaStream_t s) { return seg_sub1_head(h, s, dt1, &nodes); });
    if (!rc) rc = add_loop(1, dt1);
    if (!rc) rc = add_segment([&](cudaStream_t s) {
        int r = seg_sub1_tail(h, s, &nodes);
        return r ? r : seg_sub2_head(h, s, &nodes);
    });
    if (!rc) rc = add_loop(2, h->cfg.dt);
    if (!rc) rc = add_segment([&](cudaStream_t s) {
        int r = seg_sub2_tail(h, s, &nodes);
        return (r || !strang) ? r : seg_sub1_head(h, s, dt1, &nodes);
    });
    if (!rc && strang) rc = add_loop(1, dt1);
    if (!rc && strang) rc = add_segment([&](cudaStream_t s) { return seg_sub1_tail(h, s, &nodes); });
    if (rc) {
        cudaGraphDestroy(g);
        return rc;
    }
    cudaGraphExec_t x = nullptr;
    cudaError_t ce = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    GCK(ce);
    h->step_exec[h->cur] = x;
    h->step_graph_nodes[h->cur] = nodes;
    return PIC_OK;
}

// nsteps steps as graph launches; counts and status read back once at the end
static int step_graphs(pic_handle *h, int nsteps, long long *s1, long long *s2)
{
    int rc;
    if (!h->d_count) {
        if ((rc = dalloc(h, &h->d_count, 2))) return rc;
        GCK(cudaMallocHost((void **)&h->h_count, 2 * sizeof(int)));
    }
    GCK(cudaMemsetAsync(h->d_count, 0, 2 * sizeof(int), h->stream));
    for (int n = 0; n < nsteps; ++n) {
        if (!h->step_exec[h->cur] && (rc = build_step_graph(h))) return rc;
        GCK(cudaGraphLaunch(h->step_exec[h->cur], h->stream));
        h->launches += h->step_graph_nodes[h->cur];
        ++h->steps_done;
        if (h->cfg.sort_every > 0 && h->steps_done % h->cfg.sort_every == 0)
            if ((rc = sort_markers(h))) return rc;
    }
    GCK(cudaMemcpyAsync(h->h_count, h->d_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if ((rc = read_ctrl(h))) return rc;
    *s1 = h->h_count[0];
    *s2 = h->h_count[1];
    h->launches += 2 * (*s1 + *s2);
    h->marker_sweeps += *s1 * h->np;
    for (int which = 1; which <= 2; ++which)
        if ((rc = check_status(h, which))) return rc;
    return PIC_OK;
}

extern "C" int pic_step(pic_handle *h, int32_t nsteps, int64_t *iters_I, int64_t *iters_II)
{
    if (!h) return PIC_ERR_INVALID;
    if (nsteps < 0) return fail(h, PIC_ERR_INVALID, "nsteps < 0");
    long long s1 = 0, s2 = 0;
    int rc = PIC_OK;
    for (int n = 0; n < nsteps; ++n) {
        // graph steps once a host-loop step has opted the kernels in to their shared memory
        if (h->host_steps > 0 && graph_eligible(h)) {
            long long g1 = 0, g2 = 0;
            rc = step_graphs(h, nsteps - n, &g1, &g2);
            s1 += g1;
            s2 += g2;
            break;
        }
        int i1 = 0, i2 = 0, i3 = 0;
        if (h->cfg.splitting == PIC_SPLIT_STRANG) {
            if ((rc = substep1(h, &i1, 0.5 * h->cfg.dt))) break;
            if ((rc = substep2(h, &i2))) break;
            if ((rc = substep1(h, &i3, 0.5 * h->cfg.dt))) break;
        } else {
            if ((rc = substep1(h, &i1, h->cfg.dt))) break;
            if ((rc = substep2(h, &i2))) break;
            if (h->cfg.hbar != 0.0 && (rc = substep3(h))) break;
        }
        s1 += i1 + i3;
        s2 += i2;
        ++h->steps_done;
        ++h->host_steps;
        if (h->cfg.sort_every > 0 && h->steps_done % h->cfg.sort_every == 0)
            if ((rc = sort_markers(h))) break;
    }
    if (iters_I) *iters_I = s1;
    if (iters_II) *iters_II = s2;
    if (rc) return rc;
    return sync(h);
}

// ------------------------------------------------------------------ diagnostics
extern "C" int pic_energy(pic_handle *h, double out[7])
{
    if (!h || !out) return h ? fail(h, PIC_ERR_INVALID, "out is NULL") : PIC_ERR_INVALID;
    int rc;
    CK(cudaMemsetAsync(h->diag, 0, 8 * sizeof(double), h->stream));
    if ((rc = deposit_charge(h, h->rho))) return rc;
    DiagArgs a{};
    a.M = h->M; a.K = h->K; a.fp32 = h->fp32; a.np = h->np; a.dx = h->dx; a.w = h->cfg.weight;
    a.P = cur_parts(h);
    a.c0 = h->ay; a.c1 = h->az; a.acc = h->diag;
    launch_kinetic(a, particle_grid(h), 256, h->stream);
    CKL_N("launch_kinetic");
    if (h->cfg.hbar != 0.0) {
        if (launch_spin_energy(spin_args(h), particle_grid(h), h->stream)) return fail(h, PIC_ERR_INVALID, "bad degree");
        CKL_N("launch_spin_energy");
    }
    // split runs: the marker sums of every process (charge, kinetic, Zeeman)
    if ((rc = reduce(h, PIC_REDUCE_SUM, h->rho, h->M)) || (rc = reduce(h, PIC_REDUCE_SUM, h->diag, 1)) ||
        (rc = reduce(h, PIC_REDUCE_SUM, h->diag + 6, 1)))
        return rc;
    launch_energy_grid(h->M, h->K, h->dx, h->d_rowM0, h->d_rowM1, h->d_rowK, h->ex, h->ey, h->ez,
                       h->ay, h->az, h->rho, h->diag, h->stream);
    CKL_N("launch_energy_grid");
    double d[8];
    CK(cudaMemcpyAsync(d, h->diag, sizeof(d), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out[0] = d[0];
    out[1] = d[1];
    out[2] = d[2];
    out[3] = d[3];
    out[6] = h->cfg.hbar != 0.0 ? h->cfg.hbar * d[6] : 0.0;
    out[4] = d[0] + d[1] + d[2] + d[3] + out[6];
    out[5] = d[5];
    return PIC_OK;
}

extern "C" int pic_get_state(pic_handle *h, const pic_arrays *o, int32_t mem)
{
    if (!h || !o) return h ? fail(h, PIC_ERR_INVALID, "out is NULL") : PIC_ERR_INVALID;
    if (mem != PIC_MEM_HOST && mem != PIC_MEM_DEVICE) return fail(h, PIC_ERR_INVALID, "bad mem");
    const size_t np = (size_t)h->np, M = (size_t)h->M;
    const bool host = mem == PIC_MEM_HOST;
    // page-locked host arrays: written in caller order over the host link by one
    // kernel, through the inverse of the markers' permutation (in the other marker copy)
    double *px = (host && o->x) ? static_cast<double *>(const_cast<void *>(pinned_device_ptr(o->x))) : nullptr;
    double *pp = (host && o->p) ? static_cast<double *>(const_cast<void *>(pinned_device_ptr(o->p))) : nullptr;
    if ((o->x || o->p) && (!o->x || px) && (!o->p || pp)) {
        int32_t *inv = reinterpret_cast<int32_t *>(h->Pblk[1 - h->cur]);
        launch_store_ordered(h->fp32, h->np, h->dx, cur_parts(h), inv, px, pp, particle_grid(h), 256, h->stream);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(h, PIC_ERR_CUDA, "get_state: %s", cudaGetErrorString(e));
        h->launches += 2;
    } else if (o->x || o->p) {
        double *dx_out = o->x, *dp_out = o->p;
        // the store writes each marker to its input position (a permutation after the
        // sorts): scattered there in device memory, then copied to the host in bulk
        if (host) stage_doubles(h, 1 - h->cur, o->x ? &dx_out : nullptr, o->p ? &dp_out : nullptr);
        launch_store(h->fp32, h->np, h->dx, cur_parts(h), dx_out, dp_out, particle_grid(h), 256, h->stream);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && host) {
            if (o->x) e = cudaMemcpyAsync(o->x, dx_out, np * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess && o->p)
                e = cudaMemcpyAsync(o->p, dp_out, np * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            cudaError_t e2 = cudaStreamSynchronize(h->stream);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) return fail(h, PIC_ERR_CUDA, "get_state: %s", cudaGetErrorString(e));
        ++h->launches;
    }
    const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    struct { double *dst; const double *src; } g[] = {
        {o->ex, h->ex}, {o->ey, h->ey}, {o->ez, h->ez}, {o->ay, h->ay}, {o->az, h->az}};
    for (auto &f : g)
        if (f.dst) CK(cudaMemcpyAsync(f.dst, f.src, M * sizeof(double), kind, h->stream));
    if (h->cfg.hbar != 0.0) {
        struct { double *dst; const double *src; } sp[] = {{o->sx, h->spx}, {o->sy, h->spy}, {o->sz, h->spz}};
        for (auto &f : sp)
            if (f.dst) CK(cudaMemcpyAsync(f.dst, f.src, np * sizeof(double), kind, h->stream));
    }
    return sync(h);
}

extern "C" int pic_deposit(pic_handle *h, int32_t kind, const double *aux, double *out)
{
    if (!h) return PIC_ERR_INVALID;
    if (!out) return fail(h, PIC_ERR_INVALID, "out is NULL");
    int rc;
    if (kind == PIC_DEP_CHARGE) {
        if ((rc = deposit_charge(h, out))) return rc;
        return sync(h);
    }
    if (kind == PIC_DEP_CURRENT) {
        if (!aux) return fail(h, PIC_ERR_INVALID, "CURRENT needs the displacements");
        CK(cudaMemsetAsync(out, 0, sizeof(double) * h->M, h->stream));
        launch_ctrl_reset(h->ctrl, h->stream);
        CKL_N("launch_ctrl_reset");
        CurrentArgs a{};
        a.M = h->M; a.H = h->H; a.Dlim = h->Dlim; a.K = h->K; a.fp32 = h->fp32; a.np = h->np;
        a.dx = h->dx; a.w = h->cfg.weight; a.P = cur_parts(h); a.disp = aux; a.out = out; a.ctrl = h->ctrl;
        if (launch_current(a, particle_grid(h), 256, charge_smem(h->M, h->H), h->stream))
            return fail(h, PIC_ERR_INVALID, "bad degree");
        CKL_N("launch_current");
        if ((rc = read_ctrl(h))) return rc;
        if (h->h_ctrl->status & STATUS_NUMERIC)
            return fail(h, PIC_ERR_NUMERIC, "displacement beyond the halo or not finite");
        return PIC_OK;
    }
    if (kind == PIC_DEP_SUSCEPT) {
        if (!aux) return fail(h, PIC_ERR_INVALID, "SUSCEPT needs a*");
        CK(cudaMemsetAsync(out, 0, sizeof(double) * 2 * h->M, h->stream));
        Sweep2Args a{};
        a.status = &h->ctrl->status;
        a.M = h->M; a.H = h->H; a.K = h->K; a.fp32 = h->fp32; a.acc = h->acc; a.np = h->np; a.w = h->cfg.weight;
        a.P = cur_parts(h);
        a.an_y = h->ay; a.an_z = h->az; a.ak_y = aux; a.ak_z = aux + h->M;
        a.s_y = out; a.s_z = out + h->M;
        if (launch_sweep2(a, h->sweep_grid, h->sweep_block, h->smem2, h->stream))
            return fail(h, PIC_ERR_INVALID, "bad degree");
        CKL_N("launch_sweep2");
        return sync(h);
    }
    return fail(h, PIC_ERR_INVALID, "unknown deposit kind %d", kind);
}

extern "C" int pic_gather(pic_handle *h, int32_t field, double *out)
{
    if (!h) return PIC_ERR_INVALID;
    if (!out) return fail(h, PIC_ERR_INVALID, "out is NULL");
    if (field == PIC_FIELD_EX_PATHAVG) {
        launch_ctrl_reset(h->ctrl, h->stream);
        CKL_N("launch_ctrl_reset");
        DiagArgs a{};
        a.M = h->M; a.K = h->K; a.fp32 = h->fp32; a.np = h->np; a.dx = h->dx; a.w = h->cfg.weight;
        a.P = cur_parts(h);
        a.c0 = h->ex;
        a.out = out;
        a.Dlim = h->Dlim;
        a.status = &h->ctrl->status;
        if (launch_gather_path(a, particle_grid(h), 256, h->stream)) return fail(h, PIC_ERR_INVALID, "bad degree");
        CKL_N("launch_gather_path");
        int rc;
        if ((rc = read_ctrl(h))) return rc;
        if (h->h_ctrl->status & STATUS_NUMERIC)
            return fail(h, PIC_ERR_NUMERIC, "path gather: displacement beyond the halo or not finite");
        return PIC_OK;
    }
    const double *coef = nullptr;
    int d = h->K;
    switch (field) {
    case PIC_FIELD_EX: coef = h->ex; d = h->K - 1; break;
    case PIC_FIELD_EY: coef = h->ey; break;
    case PIC_FIELD_EZ: coef = h->ez; break;
    case PIC_FIELD_AY: coef = h->ay; break;
    case PIC_FIELD_AZ: coef = h->az; break;
    default: return fail(h, PIC_ERR_INVALID, "unknown field %d", field);
    }
    DiagArgs a{};
    a.M = h->M; a.K = h->K; a.fp32 = h->fp32; a.np = h->np; a.dx = h->dx; a.w = h->cfg.weight;
    a.P = cur_parts(h);
    a.c0 = coef;
    a.out = out;
    if (launch_gather(a, d, particle_grid(h), 256, h->stream)) return fail(h, PIC_ERR_INVALID, "bad degree");
    CKL_N("launch_gather");
    return sync(h);
}

extern "C" int pic_set_warm_mlp(pic_handle *h, pic_mlp *m)
{
    if (!h) return PIC_ERR_INVALID;
    if (h->mlp != m) drop_graphs(h);
    h->mlp = m;
    return PIC_OK;
}

extern "C" int pic_timing_enable(pic_handle *h, int32_t on)
{
    if (!h) return PIC_ERR_INVALID;
    int rc;
    if ((rc = timing_fold(h))) return rc;      // pairs of an earlier period are dropped below
    h->timing = on ? 1 : 0;
    h->t_sw1 = h->t_sw2 = h->t_solve = h->t_warm = 0.0;
    h->n_warm = 0;
    h->n_sw1 = h->n_sw2 = h->n_solve = 0;
    h->launches = 0;
    h->marker_sweeps = 0;
    return PIC_OK;
}

extern "C" int pic_timing_read(pic_handle *h, double out[10])
{
    if (!h || !out) return PIC_ERR_INVALID;
    int rc;
    if ((rc = timing_fold(h))) return rc;
    out[0] = h->t_sw1;
    out[1] = (double)h->n_sw1;
    out[2] = h->t_sw2;
    out[3] = (double)h->n_sw2;
    out[4] = h->t_solve;
    out[5] = (double)h->n_solve;
    out[6] = (double)h->launches;
    out[7] = (double)h->marker_sweeps;
    out[8] = h->t_warm;
    out[9] = (double)h->n_warm;
    return PIC_OK;
}

extern "C" int pic_destroy(pic_handle *h)
{
    if (!h) return PIC_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return PIC_OK;
}

extern "C" const char *pic_last_error(const pic_handle *h)
{
    if (!h) return g_init_error.c_str();
    return h->err.c_str();
}

extern "C" const char *pic_version(void) { return kVersion; }
