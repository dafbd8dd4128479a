// pic_handle.h -- the state behind a pic_handle (private to libpic).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "pic.h"
#include "pic_internal.h"

using pic::PartPtrs;
using pic::DevCtrl;
using pic::kSweepThreads;
using pic::StageImages;

struct pic_handle {
    pic_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int M = 0, K = 0, H = 0, Dlim = 0, fp32 = 0;
    int acc = 0;                    // deposit window accumulator of the sweeps (pic::ACC_*)
    long long np = 0;
    double dx = 0.0;
    size_t rsize = 8;               // bytes of one particle real
    long long steps_done = 0;

    // marker state: two copies of (cell, t, p, id) for the counting sort
    PartPtrs P[2]{};
    // one device block per copy holds its four arrays; between sorts the copy not
    // in use (P[1 - cur]) is free, and the host transfers stage doubles in it
    char *Pblk[2] = {nullptr, nullptr};
    int cur = 0;
    void *delta = nullptr, *pnew = nullptr;
    void *a0 = nullptr;             // subsystem-I start-point cache (4 reals a marker; FP64 form)
    // spin (hbar != 0, FP64 form): components in caller order, and the spin deposits
    double *spx = nullptr, *spy = nullptr, *spz = nullptr;
    double *sdy = nullptr, *sdz = nullptr;

    // split run: the markers of one plasma spread over several processes; marker
    // sums and maxima go through this reduction (NULL: all markers are here)
    pic_reduce_fn reduce = nullptr;
    void *rctx = nullptr;
    double *red = nullptr;          // 4 doubles: packed control entries

    // one step as a CUDA graph with device-ended loops (one per marker copy cur)
    cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
    int step_graph_nodes[2] = {0, 0};   // kernel nodes outside the loops
    cudaStream_t cap = nullptr;         // private capture stream
    int *d_count = nullptr;             // sweeps of subsystems I and II (graph mode)
    int *h_count = nullptr;             // pinned readback of d_count
    int host_steps = 0;                 // steps taken by host loops (the first one opts kernels in)

    // grid state (double)
    double *ex = nullptr, *ey = nullptr, *ez = nullptr, *ay = nullptr, *az = nullptr;
    double *ek = nullptr, *ebar = nullptr, *ga_y = nullptr, *ga_z = nullptr, *jb[2] = {nullptr, nullptr};
    double *eky = nullptr, *ekz = nullptr, *aky = nullptr, *akz = nullptr;
    double *by = nullptr, *bz = nullptr, *r0y = nullptr, *r0z = nullptr;
    double *sy[2] = {nullptr, nullptr}, *sz[2] = {nullptr, nullptr};
    double *rho = nullptr, *work = nullptr, *diag = nullptr;
    int32_t *counts = nullptr;

    // circulant bands and inverse taps
    double *d_rowM0 = nullptr, *d_rowM1 = nullptr, *d_rowK = nullptr, *d_rowPm = nullptr;
    double *d_tapM1 = nullptr, *d_tapP = nullptr;
    int tapM1_start = 0, tapM1_n = 0, tapP_start = 0, tapP_n = 0;

    StageImages img{};              // float staging images (FP32 form)
    pic::FieldHist fh{};            // field changes of the last solves (starting fields)
    DevCtrl *ctrl = nullptr;
    int *h_flag = nullptr;          // pinned: converged flag readback
    DevCtrl *h_ctrl = nullptr;      // pinned: full control block readback

    int sweep_grid = 0, sweep_block = kSweepThreads;
    size_t smem1 = 0, smem2 = 0;

    // timing: event pairs recorded around the timed launches, read back (and the
    // pairs reused) by pic_timing_read or when kMaxTimedLaunches are pending
    int timing = 0;
    struct Timed {
        cudaEvent_t b, e;
        int kind;                   // 0 sweep I, 1 sweep II, 2 solve, 3 warm start
    };
    std::vector<Timed> timed;       // pairs in use, in launch order
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
    double t_sw1 = 0, t_sw2 = 0, t_solve = 0;
    long long n_sw1 = 0, n_sw2 = 0, n_solve = 0, launches = 0, marker_sweeps = 0;

    double t_warm = 0;
    long long n_warm = 0;
    pic_mlp *mlp = nullptr;         // borrowed warm-start network

    std::string err;
};

namespace pic {
// marker sort of one handle (swaps its current buffer); its current marker arrays
int handle_sort(pic_handle *h);
PartPtrs handle_parts(pic_handle *h);
// the grid-side pointers of one handle (preparation and commit kernels)
RunDesc handle_desc(pic_handle *h);
}  // namespace pic
