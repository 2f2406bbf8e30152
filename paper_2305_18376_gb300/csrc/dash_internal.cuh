// Internal layout of a dash_model (the opaque handle of include/dash.h).
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <string>
#include <vector>

#include "dash.h"
#include "dash_kernels_fused.cuh"
#include "dash_kernels_p.cuh"
#include "dash_kernels_q.cuh"
#include "dash_kernels_err.cuh"
#include "dash_kernels_stream.cuh"
#include "dash_kernels_tc05.cuh"

namespace dash {
// kernel kinds for the per-kernel profiler
enum KernelKind {
    KK_BEGIN_NEW, KK_ROWMAP, KK_XV, KK_SLICES, KK_F, KK_F_REDUCE, KK_G_REDUCE, KK_PINV,
    KK_VUPDATE, KK_GAMMA, KK_FITNESS, KK_CAST, KK_C_RECOMPUTE, KK_VTILDE, KK_ROWS_FUSED,
    KK_BIG_B, KK_BIG_C, KK_QV, KK_PH_A, KK_PH_EPI, KK_PH_B, KK_EPI_U, KK_EPI_DD, KK_EPI_FIN,
    KK_EPI_SCALE,
    KK_Q_BEGIN, KK_Q_AROWS, KK_Q_Y, KK_Q_LT, KK_Q_H, KK_Q_VPART, KK_Q_V, KK_Q_PW, KK_Q_W,
    KK_Q_OUT, KK_Q_FIT, KK_QLT_QR, KK_QLT_PRE, KK_QLT_PASS, KK_QLT_TAIL,
    KK_XQ_PREP, KK_XQ_TC, KK_F_TC, KK_UTILDE, KK_XQ_WAIT, KK_XQ_BUSY, KK_FT_WAIT, KK_FT_BUSY,
    KK_QV_TF32, KK_XQ_UMMA, KK_F_UMMA, KK_FIT_LAMBDA,
    KK_XU_WAIT_P, KK_XU_WAIT_M, KK_XU_WAIT_C, KK_XU_WAIT_E, KK_XU_CYCLES,
    KK_BC_DSUM, KK_BC_DUPD, KK_BC_CHOL, KK_BC_SOLVE, KK_BC_RESID, KK_BC_GSHARE, KK_Q_PSUM,
    KK_HOST_PLAN, KK_HOST_WAIT, KK_HOST_LAUNCH, KK_COUNT
};
static const char *const kKernelNames[KK_COUNT] = {
    "k_begin_new", "k_rowmap", "k_xv", "k_slices", "k_f", "k_f_reduce", "k_g_reduce",
    "k_pinv_small", "k_vupdate", "k_gamma", "k_fitness", "k_cast", "k_c_recompute",
    "k_vqr", "k_rows_fused", "k_big_b", "k_big_c", "k_qv",
    "k_rows_fused.phase_a", "k_rows_fused.epilogue", "k_rows_fused.phase_b",
    "k_rows_fused.epilogue.u_rows", "k_rows_fused.epilogue.gram", "k_rows_fused.epilogue.finish",
    "k_rows_fused.epilogue.scale",
    "k_q_begin_new", "k_q_arows", "k_q_y", "k_q_lt", "k_q_h", "k_q_vpart", "k_q_v", "k_q_pw",
    "k_q_w", "k_q_out", "k_q_fit", "k_q_lt.qr", "k_q_lt.fp32_pass", "k_q_lt.passes",
    "k_q_lt.tail", "k_xq_bfrag", "k_xq_tc", "k_f_tc", "k_utilde", "k_xq_tc.wait", "k_xq_tc.loop",
    "k_f_tc.wait", "k_f_tc.loop", "k_qv_tf32", "k_xq_umma", "k_f_umma", "k_fit_lambda",
    "k_xq_umma.producer_wait", "k_xq_umma.mma_wait", "k_xq_umma.converter_wait", "k_xq_umma.epilogue_wait",
    "k_xq_umma.cta", "k_big_c.dsum", "k_big_c.d_update", "k_big_c.cholesky", "k_big_c.solves",
    "k_big_c.residual", "k_big_c.g_share", "k_q_psum", "host.plan", "host.wait_previous", "host.launch"};

struct Profiler {
    bool on = false;
    bool phases = false;                      // in-kernel phase clocks (level 2)
    int64_t launches_total = 0;
    int64_t launches[KK_COUNT] = {};
    double ms[KK_COUNT] = {};
    struct Mark { int kind; cudaEvent_t a, b; };
    std::vector<Mark> pending;
    std::vector<cudaEvent_t> pool;
    unsigned long long *d_phase = nullptr;   // SM cycles per fused-kernel phase
    double clock_khz = 1.0;
    int n_sm = 1;
    double q_lt_warps = 0.0;    // warps of the last profiled k_q_lt launch
    double xq_warps = 0.0, ft_warps = 0.0;   // warps of the streaming kernels' last launch
    double xu_ctas = 0.0;                     // CTAs of the last k_xq_umma launch
    double xu_conv_warps = 8.0;               // its converter warps per CTA
    double bc_warps = 0.0;                    // warps of the last k_big_c launch
    std::chrono::steady_clock::time_point t_plan0;   // start of the current batch's planning
};

constexpr int kPhaseSlots = 26;        // in-kernel cycle counters of the profiler
// device error slots: [0] timed-out waits, [1] FP64 fallback solves,
// [2] non-finite slice results, [3] this update abandoned, [4] failed index
// self-checks of the tcgen05 kernels, [5] the first failed check's code
constexpr int kErrSlots = 8;
constexpr int kCopyStreams = 2;         // streams sharing a large host-to-device append
constexpr size_t kSplitCopyBytes = 64u << 20;   // appends from this size are split
constexpr int kFBlocksMax = 1024;       // max row chunks of the F-partial kernel
constexpr int kSliceBlocksMax = 1216;   // max CTAs of the per-slice kernel (8 per SM)
constexpr bool kAutoSplit = true;       // DASH_ROWS_AUTO takes the split row pipeline
}  // namespace dash

struct dash_model {
    dash_config cfg{};
    std::string err;
    bool broken = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_meta = nullptr;    // after a batch's metadata copies (pinned buffers free)
    cudaStream_t copy_streams[dash::kCopyStreams] = {};   // parts of large host appends
    cudaEvent_t copy_ev[dash::kCopyStreams + 1] = {};
    double rtol = 0.0;
    size_t tsize = 4;                 // bytes of the product arithmetic type
    bool df_state = false;            // c, D stored as double-float pairs
    bool fused_ok = false;            // shapes the fused row kernel supports
    int n_sm = 1;
    bool gam_ok_host = false;         // mirror of the device flag (Γ nonsingular)
    // which outputs derived from the current Γ are up to date: the Cholesky
    // QR of V (R_V, R_V⁻ᵀ, Γ in double-float; the mixed path computes it at
    // the end of each update) and Γ⁺ (the FP64 path, and the general kernel
    // when a mixed update takes it)
    bool vqr_fresh = false;
    bool gamp_fresh = true;
    int64_t K = 0;                    // slices in the model
    bool v_set = false;

    // device state (FP64 masters) and derived copies
    dash::StateDev st{};
    void *VT = nullptr;               // V in the product type
    double *GP = nullptr;             // G⁺
    double *Finc = nullptr, *Ginc = nullptr, *fit = nullptr;

    // staging: rows copied in by the append calls, into one of two buffers
    // (the other may still be read by the update in flight)
    void *Xs = nullptr;               // the buffer being filled: Xs_buf[st_buf]
    void *Xs_buf[2] = {nullptr, nullptr};
    int st_buf = 0;
    cudaEvent_t buf_free[2] = {};     // after the last update that read the buffer
    bool copies_pending = false;      // split host copies the next update must wait for
    int64_t stage_cap = 0;            // rows a staging buffer holds
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

    // fused row kernel: tiles of single-segment slices, Ṽ, Γ (double-float)
    int *d_tile_s0 = nullptr, *d_tile_s1 = nullptr;
    int *h_tile_s0 = nullptr, *h_tile_s1 = nullptr;
    int n_tiles = 0;
    float *GPf = nullptr;             // R_V⁻ᵀ in FP32 (V = Q_V R_V)
    double *RV = nullptr, *Linv = nullptr;
    float *QV = nullptr;
    dash::df *Gdf = nullptr;
    double *wsp = nullptr;
    int *d_err = nullptr, *h_err = nullptr;
    // chunked path for slices the tiles cannot hold, and the finish list
    int64_t *d_ch_row0 = nullptr, *h_ch_row0 = nullptr;
    int *d_ch_n = nullptr, *d_ch_k = nullptr, *h_ch_n = nullptr, *h_ch_k = nullptr;
    int *d_fin_k = nullptr, *d_fin_c0 = nullptr, *h_fin_k = nullptr, *h_fin_c0 = nullptr;
    int n_chunks = 0, n_fin = 0;
    int64_t max_chunks = 0;
    float *dpart = nullptr;
    bool fused_active = false;        // this update runs the fused + chunked path
    // row pipeline of mode P (DASH_ROWS_*) and whether this update splits:
    // every slice through the chunked path, with the streaming tensor-core
    // kernels for P' = X Q_V and the F partials
    int row_path = 0;
    // updates launched as one CUDA graph: the launch sequence is captured
    // from the model's stream and, while its topology (kernel kinds, order,
    // copies) matches the previous update's, applied to the instantiated
    // graph as a parameter update (cudaGraphExecUpdate) instead of a new
    // instantiation
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_instantiations = 0, graph_updates = 0;
    bool split_active = false;
    uint4 *xq_frag = nullptr;         // Q_V split into MMA fragments
    int *xq_bexp = nullptr;           // power-of-two scale of those fragments
    uint32_t *Ut = nullptr;           // Ũ = U ∘ w_new as MMA fragment blocks of 16 rows
    int *xe = nullptr;                // exponent of each general row's max |x|
    // tcgen05 streaming X·Q_V (k_xq_umma): Q_V's TF32 slabs and the ring
    // depth for this J (0: the shape takes the warp-level kernel)
    float *qv_slabs = nullptr;
    int xu_nst = 0;
    int xr_nst = 0;                   // X ring depth of k_xq_umma_rq (0: Q_V does not fit)
    // autotuning of the X·Q_V pass on the first update that runs it: the
    // resident-Q_V kernel at each ring depth that fits and the streamed-slab
    // kernel, all computing the same bits; the fastest is kept
    bool autotune = true;
    bool xu_tuned = false;
    int xu_tune_n = 0;                // candidates timed
    float xu_tune_ms[8] = {};         // their times (ms), in candidate order
    int xu_tune_best = -1;            // index of the one kept
    long long wait_limit = 2000000000LL;   // cycles before a bounded device wait gives up
    int inject_wait_fault = 0;        // test hook: the next tcgen05 X·Q_V pass skips one copy
    int64_t K_prev = 0;               // slices before the last update (restored if it is dropped)
    float *Wf = nullptr;              // FP32 copy of the finished slices' new weights
    // general rows: runs of consecutive rows left to the general kernels
    int64_t *d_run_g0 = nullptr, *d_run_row0 = nullptr;
    int64_t *h_run_g0 = nullptr, *h_run_row0 = nullptr;

    // scratch
    void *P = nullptr, *U = nullptr;
    double *xn_part = nullptr;
    int64_t n_xn_max = 0;
    void *Fpart = nullptr;
    int n_fb_max = 0;
    double *Gpart = nullptr;
    int n_gb_max = 0;
    double *cross_part = nullptr;

    // constrained mode (Q): per-slice factor L_k, eigenbasis E_k and B_k^{1/2}
    // (in the scalar type: double, or double-float pairs), the carry C_k
    // (FP64), the projected data Y_k and the A rows in the product type; H and
    // the small solve results
    double *qL = nullptr, *qE = nullptr, *qBh = nullptr, *qC = nullptr;
    void *qY = nullptr, *qA = nullptr;
    double *qH = nullptr, *qWW = nullptr, *qPV = nullptr, *qPW = nullptr;
    double *qMH = nullptr, *qWWp = nullptr, *qslots = nullptr, *qfit = nullptr;
    int q_lt_max = 0, q_vslots = 0, q_out_max = 0;

    // the last update's batch, for dash_local_errors (valid until the next
    // append or update): X, its segments on the host, and error scratch
    const void *last_X = nullptr;
    std::vector<int64_t> last_ids, last_rp;
    double *err_rows = nullptr, *err_segs = nullptr;
    int64_t err_rows_cap = 0, err_segs_cap = 0;
    int64_t *re_seg_row = nullptr;    // segments of dash_rows_error
    int *re_seg_slice = nullptr;
    int64_t re_cap = 0;

    // plan of the last batch (dash_last_plan)
    int64_t plan_tile_rows = 0, plan_tile_slices = 0, plan_tiles = 0, plan_chunk_rows = 0,
            plan_general_rows = 0;

    // last update
    int64_t last_N = 0;
    bool has_last = false;

    // xx = Σ λ^age ||x||² over every absorbed row (the λ-weighted fitness'
    // denominator): folded on the host from each update's ||X_new||² once
    // the update has finished (xx ← xx_lam·xx + ||X_new||²)
    double xx = 0.0;
    bool xx_valid = false, xx_pending = false;
    double xx_lam = 0.0;
    // n_sweeps > 1 (mode P): the old helpers each extra pass starts from
    double *sw_c = nullptr, *sw_D = nullptr, *sw_F = nullptr, *sw_G = nullptr;

    dash::Profiler prof;

    std::vector<void *> allocs, host_allocs;
    bool dry = false;                      // init_alloc only counts bytes (dash_config_bytes)
    int64_t dev_bytes = 0, host_bytes = 0; // owned device / pinned host memory
};
