// pic_ensemble.cu -- batched ensembles of independent runs (C ABI in include/pic.h).
//
// Each run is an ordinary handle (pic_init), so its state, diagnostics and
// sort are the single-run ones.  The ensemble adds device tables of every
// run's kernel arguments and advances all runs with batched kernels:
//
//   prep1(all) -> WHILE{ plan, sweep1(queue), solve1(all active) }
//   -> finalize1(all), copy I(all) -> prep2(all), r0 = P^-1 b (all)
//   -> WHILE{ plan, sweep2(queue), solve2(all active) } -> copy II(all)
//
// The plan kernel rebuilds the work queue from the runs still iterating; the
// batched solve takes each run's convergence decision (Sec. 5 tolerance, as
// for a single run) and, once every active run has decided, ends the loop on
// the device through the conditional handle.  Sweep buffers alternate by each
// run's own sweep parity, read on the device, so the captured graph is valid
// for any number of sweeps.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pic.h"
#include "pic_handle.h"
#include "pic_internal.h"

using namespace pic;

struct pic_ensemble {
    cudaStream_t stream = nullptr;      // caller's stream (launches, graph)
    cudaStream_t cap = nullptr;         // private stream for graph capture
    int nruns = 0, K = 0, fp32 = 0, Mmax = 0, ntap1 = 0, ntap2 = 0, num_sms = 0;
    int use_graph = 1;
    int warm_field = 0;                 // every run starts subsystem I from a predicted field
    std::vector<pic_handle *> runs;

    // host mirrors and device copies of the per-run tables
    std::vector<RunDesc> desc;
    std::vector<Sweep1Args> a1, a1p;
    std::vector<Sweep2Args> a2;
    std::vector<ConvArgs> c1, c2, cp, c1p;
    std::vector<EnsRun> er;
    RunDesc *d_desc = nullptr;
    Sweep1Args *d_a1 = nullptr, *d_a1p = nullptr;
    Sweep2Args *d_a2 = nullptr;
    ConvArgs *d_c1 = nullptr, *d_c2 = nullptr, *d_cp = nullptr, *d_c1p = nullptr;
    EnsRun *d_er = nullptr;
    EnsQueue *d_q = nullptr;
    int *d_sweeps = nullptr, *d_status = nullptr;
    std::vector<SortRun> sorts;         // the runs due for their periodic sort (batched)
    SortRun *d_sorts = nullptr;
    int sort_grid = 1;
    int *h_buf = nullptr;               // pinned readback: sweeps (2 nruns), status (nruns), Q fields

    size_t smem1 = 0, smem2 = 0;
    int bps_max = 1;                    // resident sweep blocks per SM (launch grid = SMs x bps_max)
    int item_markers = 65536, bps = 1;  // schedule (the autotuner's choice)
    int fin_grid = 1;

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    long long loops_seen[2] = {0, 0};

    std::string err;
};

static int efail(pic_ensemble *e, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (e) e->err = buf;
    else set_thread_error(buf);
    return code;
}

#define ECK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return efail(e, PIC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

#define ELAUNCH(expr, what)                                                                    \
    do {                                                                                       \
        if (expr) return efail(e, PIC_ERR_CUDA, "%s: launch setup failed", what);              \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return efail(e, PIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_));             \
    } while (0)

template <typename T>
static int ealloc(pic_ensemble *e, T **p, size_t n)
{
    if (cudaMalloc((void **)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        return efail(e, PIC_ERR_NOMEM, "cudaMalloc of %zu bytes failed", n * sizeof(T));
    }
    return PIC_OK;
}

// ------------------------------------------------------------------ tables
// Per-run kernel arguments, in the form the single-run drivers build them, with
// the sweep buffers chosen by each run's sweep parity on the device.
static void build_tables(pic_ensemble *e)
{
    for (int r = 0; r < e->nruns; ++r) {
        pic_handle *h = e->runs[r];
        const PartPtrs P = handle_parts(h);

        e->desc[r] = handle_desc(h);

        Sweep1Args &a = e->a1[r];
        a = Sweep1Args{};
        a.M = h->M; a.H = h->H; a.Dlim = h->Dlim; a.K = h->K; a.fp32 = h->fp32; a.acc = h->acc; a.np = h->np;
        a.dx = h->dx; a.dt = h->cfg.dt; a.w = h->cfg.weight;
        a.P = P;
        a.ebar = h->ebar; a.ga_y = h->ga_y; a.ga_z = h->ga_z; a.ay = h->ay; a.az = h->az;
        a.ctrl = h->ctrl;
        a.j = h->jb[0];
        // with a predicted start the proposal is already in delta when the loop starts
        a.warm = (h->cfg.warm_start == PIC_WARM_EXPLICIT && !h->cfg.warm_field) ? 1 : 0;
        a.a0 = h->a0;
        a.graph = 1;
        a.jpair[0] = h->jb[0]; a.jpair[1] = h->jb[1];
        a.img = h->img;

        // the predicted start: the explicit proposal and its current into jb[1]
        Sweep1Args &ap = e->a1p[r];
        ap = a;
        ap.warm = h->cfg.warm_start == PIC_WARM_EXPLICIT ? 1 : 0;
        ap.graph = 0;
        ap.first = 1;
        ap.j = h->jb[1];

        ConvArgs &c = e->c1[r];
        c = ConvArgs{};
        c.M = h->M; c.d_start = h->tapM1_start; c.ntap = h->tapM1_n; c.mode = CONV_SOLVE1; c.ncomp = 1;
        c.taps = h->d_tapM1;
        c.en[0] = h->ex; c.ek[0] = h->ek; c.aux[0] = h->ebar;
        c.dt = h->cfg.dt; c.dx = h->dx; c.tol = h->cfg.tol; c.dtol = 1e-6;
        c.erel = h->cfg.warm_field ? kFieldIncrementRelPredicted : kFieldIncrementRel;
        c.max_iter = h->cfg.max_iter; c.fp32 = h->fp32; c.subsystem = 1; c.ctrl = h->ctrl;
        c.graph = 1;
        c.pair[0][0] = h->jb[0]; c.pair[0][1] = h->jb[1];
        c.cond_handle = 0;      // the ensemble ends the loop, not the run
        c.img = h->img;

        // e^(0) = e^n - M1^{-1} j^(0) from the predicted start's current
        ConvArgs &cs = e->c1p[r];
        cs = c;
        cs.mode = CONV_START1;
        cs.graph = 0;
        cs.in[0] = h->jb[1];

        Sweep2Args &b = e->a2[r];
        b = Sweep2Args{};
        b.status = &h->ctrl->status;
        b.M = h->M; b.H = h->H; b.K = h->K; b.fp32 = h->fp32; b.acc = h->acc; b.np = h->np; b.w = h->cfg.weight;
        b.P = P;
        b.an_y = h->ay; b.an_z = h->az; b.ak_y = h->aky; b.ak_z = h->akz;
        b.s_y = h->sy[0]; b.s_z = h->sz[0];
        b.graph = 1; b.ctrl = h->ctrl;
        b.sypair[0] = h->sy[0]; b.sypair[1] = h->sy[1];
        b.szpair[0] = h->sz[0]; b.szpair[1] = h->sz[1];
        b.img = h->img;

        ConvArgs &g = e->c2[r];
        g = ConvArgs{};
        g.M = h->M; g.d_start = h->tapP_start; g.ntap = h->tapP_n; g.mode = CONV_SOLVE2; g.ncomp = 2;
        g.taps = h->d_tapP;
        g.en[0] = h->ey; g.en[1] = h->ez; g.ek[0] = h->eky; g.ek[1] = h->ekz;
        g.aux[0] = h->aky; g.aux[1] = h->akz; g.an[0] = h->ay; g.an[1] = h->az;
        g.r0[0] = h->r0y; g.r0[1] = h->r0z;
        g.dt = h->cfg.dt; g.dx = h->dx; g.tol = h->cfg.tol; g.dtol = 0.0;
        g.max_iter = h->cfg.max_iter; g.fp32 = h->fp32; g.subsystem = 2; g.ctrl = h->ctrl;
        g.graph = 1;
        g.pair[0][0] = h->sy[0]; g.pair[0][1] = h->sy[1];
        g.pair[1][0] = h->sz[0]; g.pair[1][1] = h->sz[1];
        g.cond_handle = 0;
        g.img = h->img;

        ConvArgs &p = e->cp[r];
        p = ConvArgs{};
        p.M = h->M; p.d_start = h->tapP_start; p.ntap = h->tapP_n; p.mode = CONV_PLAIN; p.ncomp = 2;
        p.taps = h->d_tapP;
        p.in[0] = h->by; p.in[1] = h->bz; p.out[0] = h->r0y; p.out[1] = h->r0z;
        p.ctrl = h->ctrl;

        e->er[r].np = h->np;
        e->er[r].ctrl = h->ctrl;
    }
}

static int upload_tables(pic_ensemble *e)
{
    const size_t n = (size_t)e->nruns;
    ECK(cudaMemcpyAsync(e->d_desc, e->desc.data(), n * sizeof(RunDesc), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_a1, e->a1.data(), n * sizeof(Sweep1Args), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_a2, e->a2.data(), n * sizeof(Sweep2Args), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_c1, e->c1.data(), n * sizeof(ConvArgs), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_c2, e->c2.data(), n * sizeof(ConvArgs), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_cp, e->cp.data(), n * sizeof(ConvArgs), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_a1p, e->a1p.data(), n * sizeof(Sweep1Args), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_c1p, e->c1p.data(), n * sizeof(ConvArgs), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaMemcpyAsync(e->d_er, e->er.data(), n * sizeof(EnsRun), cudaMemcpyHostToDevice, e->stream));
    return PIC_OK;
}

// the schedule fields of the queue, read by the plan and sweep kernels at run time
static int upload_schedule(pic_ensemble *e)
{
    int v[2] = {e->item_markers, e->num_sms * e->bps};
    ECK(cudaMemcpyAsync(&e->d_q->item_markers, v, sizeof(v), cudaMemcpyHostToDevice, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
    return PIC_OK;
}

// ------------------------------------------------------------------ launches
// The loop body: plan, batched sweep, batched solve (cond = 0: no graph).
static int loop_body(pic_ensemble *e, int which, cudaStream_t s, unsigned long long cond)
{
    const int grid = e->num_sms * e->bps_max;
    ELAUNCH(launch_ens_plan(e->d_q, e->d_er, e->nruns, cond, s), "ensemble plan");
    if (which == 1) {
        ELAUNCH(launch_sweep1_ens(e->K, e->fp32, e->d_a1, e->nruns, e->d_q, grid, e->smem1, s), "ensemble sweep I");
        ELAUNCH(launch_conv_ens(e->d_c1, e->nruns, e->Mmax, 1, e->ntap1, e->d_q, e->d_sweeps, cond, s),
                "ensemble solve I");
    } else {
        ELAUNCH(launch_sweep2_ens(e->K, e->fp32, e->d_a2, e->nruns, e->d_q, grid, e->smem2, s), "ensemble sweep II");
        ELAUNCH(launch_conv_ens(e->d_c2, e->nruns, e->Mmax, 2, e->ntap2, e->d_q, e->d_sweeps, cond, s),
                "ensemble solve II");
    }
    return PIC_OK;
}

static int seg_prep1(pic_ensemble *e, cudaStream_t s)
{
    ELAUNCH(launch_prep1_ens(e->d_desc, e->nruns, e->Mmax, s), "ensemble prep I");
    if (e->warm_field) {
        // predicted start of every run: plan (all runs are iterating), the proposals
        // and their currents (work queue), e^(0) per run
        const int grid = e->num_sms * e->bps_max;
        ELAUNCH(launch_ens_plan(e->d_q, e->d_er, e->nruns, 0ull, s), "ensemble plan");
        ELAUNCH(launch_predeposit_ens(e->K, e->fp32, e->d_a1p, e->nruns, e->d_q, grid, e->smem1, s),
                "ensemble predicted start");
        ELAUNCH(launch_conv_ens(e->d_c1p, e->nruns, e->Mmax, 1, e->ntap1, e->d_q, e->d_sweeps, 0ull, s),
                "ensemble start field");
    }
    return PIC_OK;
}

static int seg_mid(pic_ensemble *e, cudaStream_t s)
{
    ELAUNCH(launch_finalize1_ens(e->fp32, e->d_desc, e->nruns, e->fin_grid, s), "ensemble finalize I");
    ELAUNCH(launch_commit_ens(e->d_desc, e->nruns, e->Mmax, 1, s), "ensemble commit I");
    ELAUNCH(launch_prep2_ens(e->d_desc, e->nruns, e->Mmax, s), "ensemble prep II");
    ELAUNCH(launch_conv_ens(e->d_cp, e->nruns, e->Mmax, 2, e->ntap2, e->d_q, e->d_sweeps, 0ull, s),
            "ensemble P solve");
    return PIC_OK;
}

static int seg_end(pic_ensemble *e, cudaStream_t s)
{
    ELAUNCH(launch_commit_ens(e->d_desc, e->nruns, e->Mmax, 2, s), "ensemble commit II");
    return PIC_OK;
}

// kernels launched per step outside the loops, and per loop sweep
static constexpr int kStepLaunches = 6, kLoopLaunches = 3, kStartLaunches = 3;

// Build the step graph: linear segments as child graphs, loops as WHILE nodes
// whose bodies are captured on the private stream.
static int build_graph(pic_ensemble *e)
{
    cudaGraph_t g = nullptr;
    ECK(cudaGraphCreate(&g, 0));
    cudaGraphNode_t prev = nullptr;
    int rc = PIC_OK;
    auto add_segment = [&](int (*seg)(pic_ensemble *, cudaStream_t)) -> int {
        cudaGraph_t child = nullptr;
        ECK(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
        const int r = seg(e, e->cap);
        cudaError_t ce = cudaStreamEndCapture(e->cap, &child);
        if (r) { if (child) cudaGraphDestroy(child); return r; }
        if (ce != cudaSuccess) return efail(e, PIC_ERR_CUDA, "capture: %s", cudaGetErrorString(ce));
        cudaGraphNode_t n = nullptr;
        ce = cudaGraphAddChildGraphNode(&n, g, prev ? &prev : nullptr, prev ? 1 : 0, child);
        cudaGraphDestroy(child);
        if (ce != cudaSuccess) return efail(e, PIC_ERR_CUDA, "child graph: %s", cudaGetErrorString(ce));
        prev = n;
        return PIC_OK;
    };
    auto add_loop = [&](int which) -> int {
        cudaGraphConditionalHandle hnd;
        ECK(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = hnd;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t n = nullptr;
        ECK(cudaGraphAddNode(&n, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        ECK(cudaStreamBeginCaptureToGraph(e->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const int r = loop_body(e, which, e->cap, (unsigned long long)hnd);
        cudaError_t ce = cudaStreamEndCapture(e->cap, &body);
        if (r) return r;
        if (ce != cudaSuccess) return efail(e, PIC_ERR_CUDA, "loop capture: %s", cudaGetErrorString(ce));
        prev = n;
        return PIC_OK;
    };
    if (!rc) rc = add_segment(seg_prep1);
    if (!rc) rc = add_loop(1);
    if (!rc) rc = add_segment(seg_mid);
    if (!rc) rc = add_loop(2);
    if (!rc) rc = add_segment(seg_end);
    if (rc) {
        cudaGraphDestroy(g);
        return rc;
    }
    cudaGraphExec_t x = nullptr;
    cudaError_t ce = cudaGraphInstantiate(&x, g, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(g);
        return efail(e, PIC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    e->graph = g;
    e->exec = x;
    return PIC_OK;
}

// One step with the loops driven from the host (one readback per sweep).
static int host_step(pic_ensemble *e)
{
    int rc;
    if ((rc = seg_prep1(e, e->stream))) return rc;
    for (int which = 1; which <= 2; ++which) {
        if (which == 2 && (rc = seg_mid(e, e->stream))) return rc;
        for (;;) {
            if ((rc = loop_body(e, which, e->stream, 0ull))) return rc;
            ECK(cudaMemcpyAsync(e->h_buf, &e->d_q->go, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
            ECK(cudaStreamSynchronize(e->stream));
            if (!e->h_buf[0]) break;
        }
    }
    return seg_end(e, e->stream);
}

static void ens_release(pic_ensemble *e)
{
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    auto f = [](void *p) { if (p) cudaFree(p); };
    f(e->d_desc); f(e->d_a1); f(e->d_a2); f(e->d_c1); f(e->d_c2); f(e->d_cp); f(e->d_er); f(e->d_q);
    f(e->d_a1p); f(e->d_c1p); f(e->d_sorts);
    f(e->d_sweeps); f(e->d_status);
    if (e->h_buf) cudaFreeHost(e->h_buf);
    if (e->cap) cudaStreamDestroy(e->cap);
    for (pic_handle *h : e->runs) pic_destroy(h);
}

// ------------------------------------------------------------------ C ABI
extern "C" int pic_ensemble_create(const pic_config *cfgs, const pic_arrays *ins, int32_t nruns, int32_t mem,
                                   int32_t use_graph, void *stream, pic_ensemble **out)
{
    if (!out) return PIC_ERR_INVALID;
    *out = nullptr;
    if (!cfgs || !ins || nruns < 1 || nruns > kEnsMaxRuns) {
        set_thread_error("ensemble: bad arguments (nruns must be 1..1024)");
        return PIC_ERR_INVALID;
    }
    for (int r = 1; r < nruns; ++r)
        if (cfgs[r].degree != cfgs[0].degree || cfgs[r].precision != cfgs[0].precision ||
            cfgs[r].warm_start != cfgs[0].warm_start || cfgs[r].warm_field != cfgs[0].warm_field) {
            set_thread_error("ensemble: runs must share degree, precision, warm start and warm_field");
            return PIC_ERR_INVALID;
        }
    if (cfgs[0].warm_start == PIC_WARM_MLP) {
        set_thread_error("ensemble: the learned warm start is not available for ensembles");
        return PIC_ERR_INVALID;
    }
    for (int r = 0; r < nruns; ++r)
        if ((cfgs[r].deposit != PIC_ACC_DEFAULT && cfgs[r].deposit != PIC_ACC_COMPENSATED &&
             !(cfgs[r].precision == PIC_FP64 && cfgs[r].deposit == PIC_ACC_DOUBLE)) ||
            cfgs[r].splitting != PIC_SPLIT_LIE || cfgs[r].hbar != 0.0) {
            set_thread_error("ensemble: runs use the default deposit accumulation, Lie--Trotter steps and no spin");
            return PIC_ERR_INVALID;
        }
    pic_ensemble *e = new (std::nothrow) pic_ensemble();
    if (!e) return PIC_ERR_NOMEM;
    e->stream = (cudaStream_t)stream;
    e->nruns = nruns;
    e->use_graph = use_graph ? 1 : 0;
    e->warm_field = cfgs[0].warm_field ? 1 : 0;
    auto bail = [&](int code) {
        set_thread_error(e->err.empty() ? "pic_ensemble_create failed" : e->err.c_str());
        ens_release(e);
        delete e;
        return code;
    };
    for (int r = 0; r < nruns; ++r) {
        pic_handle *h = nullptr;
        const int rc = pic_init(&cfgs[r], &ins[r], mem, stream, &h);
        if (rc) {
            efail(e, rc, "run %d: %s", r, pic_last_error(nullptr));
            return bail(rc);
        }
        e->runs.push_back(h);
    }
    pic_handle *h0 = e->runs[0];
    e->K = h0->K;
    e->fp32 = h0->fp32;
    e->num_sms = h0->num_sms;
    long long npmax = 0;
    for (pic_handle *h : e->runs) {
        e->Mmax = std::max(e->Mmax, h->M);
        e->ntap1 = std::max(e->ntap1, h->tapM1_n);
        e->ntap2 = std::max(e->ntap2, h->tapP_n);
        e->smem1 = std::max(e->smem1, h->smem1);
        e->smem2 = std::max(e->smem2, h->smem2);
        npmax = std::max(npmax, h->np);
    }
    e->fin_grid = (int)std::min<long long>(std::max<long long>((npmax + 255) / 256, 1), 64);
    {
        const int b1 = sweep_blocks_per_sm(e->K, e->fp32, e->fp32 ? ACC_COMP : ACC_NATIVE, 1, kSweepThreads, e->smem1);
        const int b2 = sweep_blocks_per_sm(e->K, e->fp32, e->fp32 ? ACC_COMP : ACC_NATIVE, 2, kSweepThreads, e->smem2);
        e->bps_max = std::max(1, std::min(b1, b2));
        e->bps = e->bps_max;
    }
    // sort blocks a run: about four sweeps of 256 markers a block for the largest
    e->sort_grid = (int)std::min<long long>(std::max<long long>((npmax + 1023) / 1024, 1), 4LL * e->num_sms);
    const size_t n = (size_t)nruns;
    e->desc.resize(n); e->a1.resize(n); e->a2.resize(n); e->c1.resize(n); e->c2.resize(n);
    e->cp.resize(n); e->er.resize(n); e->a1p.resize(n); e->c1p.resize(n);
    int rc;
    if ((rc = ealloc(e, &e->d_desc, n)) || (rc = ealloc(e, &e->d_a1, n)) || (rc = ealloc(e, &e->d_a2, n)) ||
        (rc = ealloc(e, &e->d_c1, n)) || (rc = ealloc(e, &e->d_c2, n)) || (rc = ealloc(e, &e->d_cp, n)) ||
        (rc = ealloc(e, &e->d_er, n)) || (rc = ealloc(e, &e->d_q, 1)) || (rc = ealloc(e, &e->d_sweeps, 2 * n)) ||
        (rc = ealloc(e, &e->d_status, n)) || (rc = ealloc(e, &e->d_a1p, n)) || (rc = ealloc(e, &e->d_c1p, n)) ||
        (rc = ealloc(e, &e->d_sorts, n)))
        return bail(rc);
    if (cudaMallocHost((void **)&e->h_buf, (3 * n + 8) * sizeof(int)) != cudaSuccess) return bail(PIC_ERR_NOMEM);
    if (cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess) return bail(PIC_ERR_CUDA);
    if (cudaMemsetAsync(e->d_q, 0, sizeof(EnsQueue), e->stream) != cudaSuccess ||
        cudaMemsetAsync(e->d_sweeps, 0, 2 * n * sizeof(int), e->stream) != cudaSuccess)
        return bail(PIC_ERR_CUDA);
    if (conv_ens_optin(e->Mmax, std::max(e->ntap1, e->ntap2)))
        return bail(efail(e, PIC_ERR_CUDA, "solve kernel shared-memory opt-in failed"));
    build_tables(e);
    if ((rc = upload_tables(e)) || (rc = upload_schedule(e))) return bail(rc);
    if (e->use_graph && (rc = build_graph(e))) return bail(rc);
    *out = e;
    return PIC_OK;
}

static int ens_read_status(pic_ensemble *e, int32_t *status_out, int *first_bad)
{
    const int n = e->nruns;
    ELAUNCH(launch_ens_status(e->d_er, n, e->d_status, e->stream), "ensemble status");
    ECK(cudaMemcpyAsync(e->h_buf + 2 * n, e->d_status, n * sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
    *first_bad = -1;
    for (int r = 0; r < n; ++r) {
        const int s = e->h_buf[2 * n + r];
        int code = PIC_OK;
        if (s & STATUS_TIMEOUT) code = PIC_ERR_CUDA;
        else if (s & STATUS_NUMERIC) code = PIC_ERR_NUMERIC;
        else if (s & STATUS_NOCONV) code = PIC_ERR_NOCONVERGE;
        if (status_out) status_out[r] = code;
        if (code && *first_bad < 0) *first_bad = r;
    }
    return PIC_OK;
}

extern "C" int pic_ensemble_step(pic_ensemble *e, int32_t nsteps, int64_t *sweeps, int32_t *status)
{
    if (!e) return PIC_ERR_INVALID;
    if (nsteps < 0) return efail(e, PIC_ERR_INVALID, "nsteps < 0");
    const int n = e->nruns;
    int rc;
    ECK(cudaMemsetAsync(e->d_sweeps, 0, 2 * (size_t)n * sizeof(int), e->stream));
    for (int s = 0; s < nsteps; ++s) {
        if (e->use_graph) {
            ECK(cudaGraphLaunch(e->exec, e->stream));
        } else if ((rc = host_step(e))) {
            return rc;
        }
        // periodic marker sort of the runs due, all in one batched sort (four
        // launches instead of four per run), then fresh tables
        e->sorts.clear();
        for (pic_handle *h : e->runs) {
            ++h->steps_done;
            if (h->cfg.sort_every > 0 && h->steps_done % h->cfg.sort_every == 0) {
                SortRun r{};
                const int per = bins_per_cell(h->np, h->M);
                r.np = h->np;
                r.M = h->M;
                r.nbins = kVelBinsBase * per;
                r.taup = (float)(h->cfg.dt / h->dx * per);
                r.src = handle_parts(h);
                r.dst = h->P[1 - h->cur];
                r.dst.delta = h->delta;
                r.dst.pnew = h->pnew;
                r.counts = h->counts;
                e->sorts.push_back(r);
                h->cur = 1 - h->cur;
            }
        }
        if (!e->sorts.empty()) {
            ECK(cudaMemcpyAsync(e->d_sorts, e->sorts.data(), e->sorts.size() * sizeof(SortRun),
                                cudaMemcpyHostToDevice, e->stream));
            ELAUNCH(launch_sort_ens(e->fp32, e->d_sorts, (int)e->sorts.size(), e->sort_grid, e->stream),
                    "ensemble sort");
            e->launches += 4;
            build_tables(e);
            if ((rc = upload_tables(e))) return rc;
        }
    }
    ECK(cudaMemcpyAsync(e->h_buf, e->d_sweeps, 2 * (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaMemcpyAsync(e->h_buf + 3 * n, e->d_q->loops, 2 * sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
    if (sweeps)
        for (int i = 0; i < 2 * n; ++i) sweeps[i] += e->h_buf[i];
    {
        const long long l1 = e->h_buf[3 * n], l2 = e->h_buf[3 * n + 1];
        e->launches += (long long)nsteps * (kStepLaunches + (e->warm_field ? kStartLaunches : 0)) +
                       kLoopLaunches * ((l1 - e->loops_seen[0]) + (l2 - e->loops_seen[1]));
        e->loops_seen[0] = l1;
        e->loops_seen[1] = l2;
    }
    int bad = -1;
    if ((rc = ens_read_status(e, status, &bad))) return rc;
    if (bad >= 0) {
        const int s = e->h_buf[2 * n + bad];
        const int code = (s & STATUS_TIMEOUT) ? PIC_ERR_CUDA : (s & STATUS_NUMERIC) ? PIC_ERR_NUMERIC : PIC_ERR_NOCONVERGE;
        return efail(e, code, "run %d stopped (status bits %d)", bad, s);
    }
    return PIC_OK;
}

extern "C" int pic_ensemble_set_schedule(pic_ensemble *e, int32_t item_markers, int32_t blocks_per_sm)
{
    if (!e) return PIC_ERR_INVALID;
    if (item_markers < 1024 || item_markers % 1024 != 0 || blocks_per_sm < 1 || blocks_per_sm > e->bps_max)
        return efail(e, PIC_ERR_INVALID, "schedule: item_markers must be a positive multiple of 1024, "
                                          "blocks per SM in 1..%d", e->bps_max);
    e->item_markers = item_markers;
    e->bps = blocks_per_sm;
    return upload_schedule(e);
}

// cache key: device name and SM count, degree, precision, runs, and the grid sizes
// and marker counts rounded to powers of two
static std::string tune_key(pic_ensemble *e)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::vector<int> lm, ln;
    for (pic_handle *h : e->runs) {
        lm.push_back((int)std::lround(std::log2((double)h->M)));
        ln.push_back((int)std::lround(std::log2((double)h->np)));
    }
    std::sort(lm.begin(), lm.end());
    std::sort(ln.begin(), ln.end());
    std::string k = prop.name;
    for (char &c : k)
        if (c == ' ' || c == '\t') c = '_';
    char buf[96];
    snprintf(buf, sizeof(buf), "|sm%d|k%d|%s|n%d|", e->num_sms, e->K, e->fp32 ? "f32" : "f64", e->nruns);
    k += buf;
    for (int v : lm) k += std::to_string(v) + ",";
    k += "|";
    for (int v : ln) k += std::to_string(v) + ",";
    return k;
}

extern "C" int pic_ensemble_tune(pic_ensemble *e, const char *cache_path, int32_t choice[3])
{
    if (!e) return PIC_ERR_INVALID;
    const std::string key = tune_key(e);
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "r")) {
            char line[8192];
            int im = 0, b = 0;
            bool hit = false;
            while (fgets(line, sizeof(line), f)) {
                char *sp = strrchr(line, ' ');
                if (!sp) continue;
                // line: <key> <item_markers>,<blocks_per_sm>
                if ((size_t)(sp - line) == key.size() && strncmp(line, key.c_str(), key.size()) == 0 &&
                    sscanf(sp + 1, "%d,%d", &im, &b) == 2)
                    hit = true;
            }
            fclose(f);
            if (hit && pic_ensemble_set_schedule(e, im, b) == PIC_OK) {
                if (choice) { choice[0] = im; choice[1] = b; choice[2] = 1; }
                return PIC_OK;
            }
        }
    }
    long long np_total = 0;
    for (pic_handle *h : e->runs) np_total += h->np;
    std::vector<std::pair<int, int>> cands;
    for (int im : {16384, 65536, 262144})
        for (int b = 1; b <= e->bps_max; ++b) cands.push_back({im, b});
    cudaEvent_t t0, t1;
    ECK(cudaEventCreate(&t0));
    ECK(cudaEventCreate(&t1));
    int rc = PIC_OK;
    double best = 1e300;
    int bi = e->item_markers, bb = e->bps;
    std::vector<int64_t> sw(2 * (size_t)e->nruns);
    // one untimed step with the current schedule, then one timed step per candidate
    rc = pic_ensemble_step(e, 1, nullptr, nullptr);
    for (size_t c = 0; c < cands.size() && rc == PIC_OK; ++c) {
        if ((rc = pic_ensemble_set_schedule(e, cands[c].first, cands[c].second))) break;
        std::fill(sw.begin(), sw.end(), 0);
        cudaEventRecord(t0, e->stream);
        if ((rc = pic_ensemble_step(e, 1, sw.data(), nullptr))) break;
        cudaEventRecord(t1, e->stream);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        double work = 0.0;     // marker-sweeps of this step
        for (int r = 0; r < e->nruns; ++r) work += (double)e->runs[r]->np * (double)(sw[2 * r] + sw[2 * r + 1]);
        const double cost = work > 0 ? ms / work : 1e300;
        if (cost < best) { best = cost; bi = cands[c].first; bb = cands[c].second; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    (void)np_total;
    if (rc) return rc;
    if ((rc = pic_ensemble_set_schedule(e, bi, bb))) return rc;
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d,%d\n", key.c_str(), bi, bb);
            fclose(f);
        }
    }
    if (choice) { choice[0] = bi; choice[1] = bb; choice[2] = 0; }
    return PIC_OK;
}

extern "C" pic_handle *pic_ensemble_run(pic_ensemble *e, int32_t r)
{
    if (!e || r < 0 || r >= e->nruns) return nullptr;
    return e->runs[r];
}

extern "C" int64_t pic_ensemble_launches(const pic_ensemble *e) { return e ? e->launches : 0; }

extern "C" int pic_ensemble_destroy(pic_ensemble *e)
{
    if (!e) return PIC_OK;
    cudaStreamSynchronize(e->stream);
    ens_release(e);
    delete e;
    return PIC_OK;
}

extern "C" const char *pic_ensemble_last_error(const pic_ensemble *e)
{
    if (!e) return pic_last_error(nullptr);
    return e->err.c_str();
}
