// Host-side plumbing shared by the translation units of the library: error
// reporting, the launch macro (launch counting and optional per-kernel
// events) and the per-mode update entry points.
#pragma once
#include <cuda_runtime.h>

#include "dash.h"
#include "dash_internal.cuh"

namespace dash {
// Record an error message on the model and return s.
dash_status fail(dash_model *m, dash_status s, const char *fmt, ...);
// An event from the model's profiler pool.
cudaEvent_t prof_event(dash_model *m);

// Mode P (Algorithm 1): one update of the planned batch; and c_k from the
// final factors at the end of a static fit (Eq. 6).
dash_status run_update_p(dash_model *m, const BatchDev &b, const void *X, double lam, bool begin_new);
dash_status recompute_c(dash_model *m, const BatchDev &b, const void *X);
// Mode Q: one update (sweep) or the summaries of the current factors alone.
dash_status run_update_q(dash_model *m, const BatchDev &b, const void *X, double lam, bool begin_new,
                         bool sweep);
// Mode Q: the eigenbasis and B_k^{1/2} of every slice from a loaded L_k.
dash_status prepare_q(dash_model *m);
}  // namespace dash

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            m->broken = true;                                                            \
            return fail(m, DASH_ECUDA, "%s failed: %s (%s:%d)", #call,                   \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                     \
        }                                                                                \
    } while (0)

#define CKL()                                                                            \
    do {                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess) {                                                         \
            m->broken = true;                                                            \
            return fail(m, DASH_ECUDA, "kernel launch failed: %s (%s:%d)",               \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                     \
        }                                                                                \
    } while (0)

// Launch a kernel on the model's stream; with profiling on, bracket it with
// events.  Every launch is counted.
#define LAUNCH(kind, ...)                                                                \
    do {                                                                                 \
        cudaEvent_t a_ = nullptr;                                                        \
        if (m->prof.on) {                                                                \
            a_ = prof_event(m);                                                          \
            cudaEventRecord(a_, m->stream);                                              \
        }                                                                                \
        __VA_ARGS__;                                                                     \
        CKL();                                                                           \
        m->prof.launches_total += 1;                                                     \
        if (m->prof.on) {                                                                \
            cudaEvent_t b_ = prof_event(m);                                              \
            cudaEventRecord(b_, m->stream);                                              \
            m->prof.pending.push_back({(int)(kind), a_, b_});                            \
        }                                                                                \
    } while (0)

namespace dash {
// Launch the R×R PSD pseudo-inverse (G⁺ or Γ⁺) on the model's stream: the
// column-parallel Cholesky kernel for R <= 32, the one-warp kernel above.
// abandoned (may be null): see k_f_reduce.
inline dash_status launch_pinv(dash_model *m, const double *in, double *out, int *ok,
                               const int *abandoned) {
    const int R = m->cfg.R;
    const size_t psm = (size_t)(3 * R * (R + 1) + (R + 1)) * 8;
    if (R <= 32)
        LAUNCH(KK_PINV, k_pinv_cols<<<R, 32, psm, m->stream>>>(in, R, m->rtol, out, ok, abandoned));
    else
        LAUNCH(KK_PINV, k_pinv_small<<<1, 32, psm, m->stream>>>(in, R, m->rtol, out, ok, abandoned));
    return DASH_OK;
}
}  // namespace dash
