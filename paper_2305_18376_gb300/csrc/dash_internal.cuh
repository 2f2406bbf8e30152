// Internal layout of a dash_model (the opaque handle of include/dash.h).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dash.h"
#include "dash_kernels_p.cuh"

namespace dash {
constexpr int kFBlocksMax = 1024;       // max row chunks of the F-partial kernel
constexpr int kSliceBlocksMax = 1216;   // max CTAs of the per-slice kernel (8 per SM)
}  // namespace dash

struct dash_model {
    dash_config cfg{};
    std::string err;
    bool broken = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double rtol = 0.0;
    size_t tsize = 4;                 // bytes of the product arithmetic type
    int64_t K = 0;                    // slices in the model
    bool v_set = false;

    // device state (FP64 masters) and derived copies
    dash::StateDev st{};
    void *VT = nullptr;               // V in the product type
    double *GP = nullptr;             // G⁺
    double *Finc = nullptr, *Ginc = nullptr, *fit = nullptr;

    // staging: rows copied in by the append calls
    void *Xs = nullptr;
    int64_t st_rows = 0, st_new = 0;
    std::vector<int64_t> st_slice;    // slice id per staged segment
    std::vector<int64_t> st_row{0};   // row offsets, size = segments + 1
    int64_t st_segs() const { return (int64_t)st_slice.size(); }

    // batch metadata (device) and their pinned host sources
    int *d_seg_slice = nullptr, *d_tslot = nullptr, *d_tseg_ptr = nullptr, *d_tseg_idx = nullptr;
    int64_t *d_seg_row = nullptr;
    int *d_row_slice = nullptr;
    int *h_seg_slice = nullptr, *h_tslot = nullptr, *h_tseg_ptr = nullptr, *h_tseg_idx = nullptr;
    int64_t *h_seg_row = nullptr;
    double *h_fit = nullptr;

    // scratch
    void *P = nullptr, *U = nullptr;
    double *xn_part = nullptr;
    int64_t n_xn_max = 0;
    void *Fpart = nullptr;
    int n_fb_max = 0;
    double *Gpart = nullptr;
    int n_gb_max = 0;
    double *cross_part = nullptr;

    // last update
    int64_t last_N = 0;
    bool has_last = false;

    std::vector<void *> allocs, host_allocs;
};
