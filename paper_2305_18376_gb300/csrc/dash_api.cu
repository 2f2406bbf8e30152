// C ABI of the Dash library (include/dash.h): model life cycle, staging of
// new rows, per-update planning on the host, and the launch sequence of one
// update on the model's CUDA stream.
#include <cuda_runtime.h>

#include <chrono>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "dash.h"
#include "dash_host.cuh"
#include "dash_internal.cuh"

using namespace dash;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
dash_status dash::fail(dash_model *m, dash_status s, const char *fmt, ...) {
    if (m) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        m->err = buf;
    }
    return s;
}

// ---------------------------------------------------------------------------
// launch accounting and the optional per-kernel profiler
// ---------------------------------------------------------------------------
cudaEvent_t dash::prof_event(dash_model *m) {
    if (!m->prof.pool.empty()) {
        cudaEvent_t e = m->prof.pool.back();
        m->prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void prof_collect(dash_model *m) {
    if (m->prof.pending.empty()) return;
    cudaStreamSynchronize(m->stream);
    for (auto &mk : m->prof.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) {
            m->prof.ms[mk.kind] += ms;
            m->prof.launches[mk.kind] += 1;
        }
        m->prof.pool.push_back(mk.a);
        m->prof.pool.push_back(mk.b);
    }
    m->prof.pending.clear();
    if (m->prof.d_phase) {
        unsigned long long c[kPhaseSlots] = {};
        if (cudaMemcpy(c, m->prof.d_phase, sizeof c, cudaMemcpyDeviceToHost) == cudaSuccess) {
            // phases: average per SM; epilogue sub-phases: average per warp;
            // milliseconds at the device clock
            for (int i = 0; i < 7; ++i) {
                const double per = i < 3 ? m->prof.n_sm : (double)m->prof.n_sm * FU_WARPS;
                m->prof.ms[KK_PH_A + i] += (double)c[i] / per / m->prof.clock_khz;
                if (c[i]) m->prof.launches[KK_PH_A + i] += 1;
            }
            // k_q_lt sub-phases: summed over its warps, reported per warp
            for (int i = 0; i < 4; ++i) {
                const double per = m->prof.q_lt_warps > 0 ? m->prof.q_lt_warps : 1.0;
                m->prof.ms[KK_QLT_QR + i] += (double)c[7 + i] / per / m->prof.clock_khz;
                if (c[7 + i]) m->prof.launches[KK_QLT_QR + i] += 1;
            }
            // streaming kernels: cycles waiting on / computing stages, summed
            // over their warps, reported per warp
            for (int i = 0; i < 4; ++i) {
                const double w = i < 2 ? m->prof.xq_warps : m->prof.ft_warps;
                m->prof.ms[KK_XQ_WAIT + i] += (double)c[11 + i] / (w > 0 ? w : 1.0) / m->prof.clock_khz;
                if (c[11 + i]) m->prof.launches[KK_XQ_WAIT + i] += 1;
            }
            // k_xq_umma: cycles each role waited (producer and MMA issuer: one
            // thread per CTA; converters and epilogue: summed over their
            // warps) and each CTA's lifetime, reported per CTA
            for (int i = 0; i < 5; ++i) {
                const double nw = i == 2 ? m->prof.xu_conv_warps : (i == 3 ? 4.0 * XU_EPI_GROUPS : 1.0);
                const double per = (m->prof.xu_ctas > 0 ? m->prof.xu_ctas : 1.0) * nw;
                m->prof.ms[KK_XU_WAIT_P + i] += (double)c[15 + i] / per / m->prof.clock_khz;
                if (c[15 + i]) m->prof.launches[KK_XU_WAIT_P + i] += 1;
            }
            // k_big_c: cycles per phase of the slice finish, summed over its
            // warps, reported per warp
            for (int i = 0; i < 6; ++i) {
                const double per = m->prof.bc_warps > 0 ? m->prof.bc_warps : 1.0;
                m->prof.ms[KK_BC_DSUM + i] += (double)c[20 + i] / per / m->prof.clock_khz;
                if (c[20 + i]) m->prof.launches[KK_BC_DSUM + i] += 1;
            }
            cudaMemset(m->prof.d_phase, 0, sizeof c);
        }
    }
    cudaGetLastError();
}

extern "C" int64_t dash_launch_count(const dash_model *m) {
    return m ? m->prof.launches_total : -1;
}

extern "C" dash_status dash_profile_enable(dash_model *m, int32_t on) {
    if (!m) return DASH_EINVAL;
    if (!m->prof.d_phase) {
        void *p = nullptr;
        if (cudaMalloc(&p, kPhaseSlots * sizeof(unsigned long long)) == cudaSuccess) {
            m->prof.d_phase = (unsigned long long *)p;
            m->allocs.push_back(p);
            cudaMemset(p, 0, kPhaseSlots * sizeof(unsigned long long));
            int dev = 0, khz = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
            m->prof.clock_khz = khz > 0 ? khz : 1.0;
            m->prof.n_sm = m->n_sm;
        }
        cudaGetLastError();
    }
    if (on < 0 || on > 2) return fail(m, DASH_EINVAL, "profiling level must be 0, 1 or 2");
    prof_collect(m);
    m->prof.on = on != 0;
    m->prof.phases = on == 2;
    for (int i = 0; i < KK_COUNT; ++i) {
        m->prof.ms[i] = 0.0;
        m->prof.launches[i] = 0;
    }
    return DASH_OK;
}

extern "C" int32_t dash_profile_kinds(void) { return KK_COUNT; }

extern "C" dash_status dash_counters(const dash_model *mc, int64_t *timeouts, int64_t *fallbacks) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    int h[4] = {0, 0, 0, 0};
    CK(cudaStreamSynchronize(m->stream));
    CK(cudaMemcpy(h, m->d_err, sizeof h, cudaMemcpyDeviceToHost));
    if (timeouts) *timeouts = h[0];
    if (fallbacks) *fallbacks = h[1];
    return DASH_OK;
}

extern "C" dash_status dash_profile_get(const dash_model *mc, int32_t i, const char **name,
                                        int64_t *launches, double *total_ms) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m || i < 0 || i >= KK_COUNT) return DASH_EINVAL;
    prof_collect(m);
    if (name) *name = kKernelNames[i];
    if (launches) *launches = m->prof.launches[i];
    if (total_ms) *total_ms = m->prof.ms[i];
    return DASH_OK;
}

extern "C" const char *dash_status_string(dash_status s) {
    switch (s) {
    case DASH_OK: return "ok";
    case DASH_EINVAL: return "invalid argument";
    case DASH_ENOMEM: return "out of memory or capacity";
    case DASH_ECUDA: return "CUDA error";
    case DASH_ESTATE: return "invalid state";
    case DASH_ENUMERIC: return "non-finite result";
    case DASH_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

extern "C" const char *dash_last_error(const dash_model *m) {
    return m ? m->err.c_str() : "null model";
}

extern "C" void dash_config_default(dash_config *cfg, int32_t J, int32_t R, double lambda) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->J = J;
    cfg->R = R;
    cfg->lambda = lambda;
    cfg->mode = DASH_MODE_P;
    cfg->precision = DASH_PREC_FP32;
    cfg->input_dtype = DASH_F32;
    cfg->n_sweeps = 1;
    cfg->pinv_rtol = 0.0;
    cfg->max_slices = 1 << 16;
    cfg->max_rows = 1 << 20;
    cfg->max_segments = 1 << 17;
    cfg->stream = nullptr;
    cfg->max_staged_rows = 0;
}

// ---------------------------------------------------------------------------
// allocation helpers
// ---------------------------------------------------------------------------
// cudaMalloc's granularity for the footprint accounting
static int64_t alloc_rounded(size_t bytes) { return (int64_t)((bytes + 511) / 512 * 512); }

static dash_status dalloc(dash_model *m, void **p, size_t bytes, const char *what) {
    if (bytes == 0) bytes = 16;
    m->dev_bytes += alloc_rounded(bytes);
    if (m->dry) {
        *p = nullptr;
        return DASH_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(m, DASH_ENOMEM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what,
                    cudaGetErrorString(e));
    }
    m->allocs.push_back(*p);
    return DASH_OK;
}

#define DALLOC(ptr, bytes, what)                                                         \
    do {                                                                                 \
        dash_status s_ = dalloc(m, (void **)&(ptr), (bytes), (what));                    \
        if (s_ != DASH_OK) return s_;                                                    \
    } while (0)

static void free_all(dash_model *m) {
    for (void *p : m->allocs) cudaFree(p);
    m->allocs.clear();
    for (void *p : m->host_allocs) cudaFreeHost(p);
    m->host_allocs.clear();
}

static dash_status halloc(dash_model *m, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    m->host_bytes += alloc_rounded(bytes);
    if (m->dry) {
        *p = nullptr;
        return DASH_OK;
    }
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(m, DASH_ENOMEM, "cudaMallocHost of %zu bytes failed", bytes);
    }
    m->host_allocs.push_back(*p);
    return DASH_OK;
}

static dash_status init_alloc(dash_model *m) {
    const dash_config &c = m->cfg;
    const int64_t J = c.J, R = c.R, Km = c.max_slices, Nm = c.max_rows, Sm = c.max_segments;
    const size_t te = m->tsize;
    const size_t ie = (c.input_dtype == DASH_F64) ? 8 : 4;
    // state
    DALLOC(m->st.V, J * R * 8, "V");
    DALLOC(m->st.W, Km * R * 8, "W");
    DALLOC(m->st.F, J * R * 8, "F");
    DALLOC(m->st.G, R * R * 8, "G");
    DALLOC(m->st.Gam, R * R * 8, "Gamma");
    DALLOC(m->st.GamP, R * R * 8, "Gamma+");
    DALLOC(m->st.gam_ok, sizeof(int), "flag");
    DALLOC(m->VT, J * R * te, "V (compute type)");
    DALLOC(m->GP, R * R * 8, "G+");
    DALLOC(m->Finc, J * R * 8, "F_inc");
    DALLOC(m->Ginc, R * R * 8, "G_inc");
    DALLOC(m->fit, 6 * 8, "fitness");       // batch fitness [4], λ-weighted fitness [2]
    if (c.mode == DASH_MODE_P) {
        DALLOC(m->st.c, Km * R * 8, "c");
        DALLOC(m->st.D, Km * R * R * 8, "D");
        if (c.n_sweeps > 1) {
            DALLOC(m->sw_c, Km * R * 8, "c (sweep start)");
            DALLOC(m->sw_D, Km * R * R * 8, "D (sweep start)");
            DALLOC(m->sw_F, J * R * 8, "F (sweep start)");
            DALLOC(m->sw_G, R * R * 8, "G (sweep start)");
        }
    } else {
        DALLOC(m->qL, Km * R * R * 8, "L_k");
        DALLOC(m->qE, Km * R * R * 8, "E_k");
        DALLOC(m->qBh, Km * R * R * 8, "B_k^1/2");
        DALLOC(m->qC, Km * R * R * 8, "carry C_k");
        DALLOC(m->qY, (size_t)Km * R * J * te, "Y_k");
        DALLOC(m->qA, (size_t)Nm * R * te, "A_new");
        DALLOC(m->qH, R * R * 8, "H");
        DALLOC(m->qWW, R * R * 8, "W^T W");
        DALLOC(m->qPV, R * R * 8, "V-step pinv");
        DALLOC(m->qPW, R * R * 8, "W-step pinv");
        m->q_lt_max = 4 * m->n_sm;
        DALLOC(m->qMH, (size_t)m->q_lt_max * R * R * 8, "H-MTTKRP partials");
        DALLOC(m->qWWp, (size_t)m->q_lt_max * R * R * 8, "W^T W partials");
        m->q_vslots = 4 * m->n_sm;
        DALLOC(m->qslots, (size_t)m->q_vslots * J * R * 8, "V-MTTKRP slots");
        m->q_out_max = 4 * m->n_sm;
        DALLOC(m->qfit, (size_t)m->q_out_max * 2 * 8, "residual partials");
    }
    // staging and batch metadata
    m->stage_cap = c.max_staged_rows > 0 ? std::min<int64_t>(c.max_staged_rows, Nm) : Nm;
    DALLOC(m->Xs_buf[0], m->stage_cap * J * ie, "staged X");
    DALLOC(m->Xs_buf[1], m->stage_cap * J * ie, "staged X");
    m->Xs = m->Xs_buf[0];
    DALLOC(m->d_seg_slice, Sm * 4, "segment ids");
    DALLOC(m->d_seg_row, (Sm + 1) * 8, "segment rows");
    DALLOC(m->d_tslot, Km * 4, "slice slots");
    DALLOC(m->d_tseg_ptr, (Sm + 1) * 4, "slice segment ptr");
    DALLOC(m->d_tseg_idx, Sm * 4, "slice segment idx");
    DALLOC(m->d_row_slice, Nm * 4, "row slice");
    // scratch
    DALLOC(m->P, Nm * R * te, "P = X V");
    DALLOC(m->U, Nm * R * te, "U_new");
    m->n_xn_max = m->n_sm + (Nm + XV_ROWS - 1) / XV_ROWS;
    DALLOC(m->xn_part, m->n_xn_max * 8, "||X|| partials");
    m->n_fb_max = m->n_sm + kFBlocksMax;
    DALLOC(m->Fpart, (size_t)m->n_fb_max * J * R * te, "F partials");
    m->n_gb_max = m->n_sm + kSliceBlocksMax;
    DALLOC(m->Gpart, (size_t)m->n_gb_max * R * R * 8, "G partials");
    DALLOC(m->cross_part, ((J + 7) / 8) * 8, "cross partials");
    // fused row kernel and general runs
    DALLOC(m->d_tile_s0, (Sm + 1) * 4, "tiles");
    DALLOC(m->d_tile_s1, (Sm + 1) * 4, "tiles");
    DALLOC(m->GPf, R * R * 4, "R_V^-T (FP32)");
    DALLOC(m->RV, R * R * 8, "R_V");
    DALLOC(m->Linv, R * R * 8, "R_V^-T");
    DALLOC(m->QV, J * R * 4, "Q_V");
    DALLOC(m->Gdf, R * R * 8, "Gamma (double-float)");
    DALLOC(m->xq_frag, (size_t)((J + 15) / 16) * ((R + 7) / 8) * 32 * 16, "Q_V fragments");
    DALLOC(m->xq_bexp, 4, "Q_V fragment scale");
    if (m->xu_nst > 0) {
        DALLOC(m->qv_slabs, (size_t)xu_slabs((int)J) * XU_SLAB_BYTES, "Q_V TF32 slabs");
    }
    if (m->fused_ok) {
        DALLOC(m->Ut, (size_t)(Nm / 16 + 2) * ft_ublk((R + 7) / 8) * 4, "U o w fragments");
        DALLOC(m->xe, (size_t)(Nm + 16) * 4, "row exponents");
        DALLOC(m->Wf, (size_t)Km * R * 4, "w_new (FP32)");
    }
    // FP64 fallback workspace: one slot per warp of a grid of at most kBigCBlocksPerSM CTAs per SM
    DALLOC(m->wsp, (size_t)kBigCBlocksPerSM * m->n_sm * FU_WARPS * fu_wsp_doubles((int)R) * 8, "fallback workspace");
    DALLOC(m->d_err, kErrSlots * sizeof(int), "error counters");
    m->max_chunks = Nm / FU_TILE_MAX + Sm + 1;
    DALLOC(m->d_ch_row0, m->max_chunks * 8, "chunks");
    DALLOC(m->d_ch_n, m->max_chunks * 4, "chunks");
    DALLOC(m->d_ch_k, m->max_chunks * 4, "chunks");
    DALLOC(m->d_fin_k, Km * 4, "finish list");
    DALLOC(m->d_fin_c0, (Km + 1) * 4, "finish list");
    DALLOC(m->dpart, (size_t)m->max_chunks * (R * R + R) * 4, "chunk partials");
    DALLOC(m->d_run_g0, (Sm + 2) * 8, "general runs");
    DALLOC(m->d_run_row0, (Sm + 2) * 8, "general runs");

    // pinned host metadata (upload source)
    dash_status s;
    if ((s = halloc(m, (void **)&m->h_seg_slice, Sm * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_seg_row, (Sm + 1) * 8))) return s;
    if ((s = halloc(m, (void **)&m->h_tslot, Km * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_tseg_ptr, (Sm + 1) * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_tseg_idx, Sm * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_fit, 4 * 8))) return s;
    if ((s = halloc(m, (void **)&m->h_tile_s0, (Sm + 1) * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_tile_s1, (Sm + 1) * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_run_g0, (Sm + 2) * 8))) return s;
    if ((s = halloc(m, (void **)&m->h_run_row0, (Sm + 2) * 8))) return s;
    if ((s = halloc(m, (void **)&m->h_err, kErrSlots * sizeof(int)))) return s;
    if ((s = halloc(m, (void **)&m->h_ch_row0, m->max_chunks * 8))) return s;
    if ((s = halloc(m, (void **)&m->h_ch_n, m->max_chunks * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_ch_k, m->max_chunks * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_fin_k, Km * 4))) return s;
    if ((s = halloc(m, (void **)&m->h_fin_c0, (Km + 1) * 4))) return s;
    if (m->dry) return DASH_OK;
    memset(m->h_err, 0, kErrSlots * sizeof(int));
    cudaMemsetAsync(m->d_err, 0, kErrSlots * sizeof(int), m->stream);
    return DASH_OK;
}

// Validate m->cfg and derive the sizes init_alloc uses (no CUDA allocation).
static dash_status init_check(dash_model *m) {
    const dash_config &c = m->cfg;
    auto bad = [&](const char *msg) {
        fail(m, DASH_EINVAL, "%s", msg);
        return DASH_EINVAL;
    };
    dash_status st = DASH_OK;
    if (c.J <= 0) st = bad("J must be positive");
    else if (c.R < 1 || c.R > kMaxR) st = bad("R must be in 1..64");
    else if (!(c.lambda > 0.0 && c.lambda <= 1.0)) st = bad("lambda must be in (0, 1]");
    else if (c.mode != DASH_MODE_P && c.mode != DASH_MODE_Q) st = bad("unknown mode");
    else if (c.precision != DASH_PREC_FP64 && c.precision != DASH_PREC_FP32 &&
             c.precision != DASH_PREC_F16X3) st = bad("unknown precision");
    else if (c.input_dtype != DASH_F64 && c.input_dtype != DASH_F32) st = bad("unknown input dtype");
    else if (c.n_sweeps < 1 || c.n_sweeps > 64) st = bad("n_sweeps must be in 1..64");
    else if (c.n_sweeps != 1 && c.mode != DASH_MODE_P) st = bad("mode Q runs one sweep per update (n_sweeps = 1)");
    else if (c.max_slices < 1 || c.max_rows < 1 || c.max_segments < 1) st = bad("capacities must be positive");
    else if (c.max_slices > INT32_MAX / 2 || c.max_segments > INT32_MAX / 2) st = bad("capacity too large");
    if (st != DASH_OK) return st;
    m->rtol = c.pinv_rtol > 0.0 ? c.pinv_rtol : (double)c.R * DBL_EPSILON;
    m->tsize = (c.precision == DASH_PREC_FP64) ? 8 : 4;
    m->df_state = c.precision != DASH_PREC_FP64;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            m->n_sm = nsm;
        cudaGetLastError();
    }
    m->fused_ok = m->df_state && c.input_dtype == DASH_F32 && c.R <= FU_RP &&
                  c.J <= FU_WARPS * FU_JG && (c.J % 4) == 0 && c.mode == DASH_MODE_P;
    // the tcgen05 X·Q_V pass (mode P) or X·V pass (mode Q): FP32 input, mixed
    // products, R <= 32, 16-byte rows
    const bool xu_shape = c.input_dtype == DASH_F32 && c.precision == DASH_PREC_F16X3 && c.R <= 32 &&
                          (c.J % 4) == 0;
    m->xu_nst = ((m->fused_ok || c.mode == DASH_MODE_Q) && xu_shape) ? xu_stages(c.J) : 0;
    m->xr_nst = m->xu_nst > 0 ? xr_stages(c.J) : 0;
    m->st.J = c.J;
    m->st.R = c.R;
    m->st.lam = c.lambda;
    m->st.rtol = m->rtol;
    return DASH_OK;
}

extern "C" dash_status dash_config_bytes(const dash_config *cfg, int64_t *device_bytes, int64_t *host_bytes) {
    if (!cfg) return DASH_EINVAL;
    dash_model m;
    m.cfg = *cfg;
    m.dry = true;
    dash_status st = init_check(&m);
    if (st == DASH_OK) st = init_alloc(&m);
    if (st != DASH_OK) return st;
    if (device_bytes) *device_bytes = m.dev_bytes;
    if (host_bytes) *host_bytes = m.host_bytes;
    return DASH_OK;
}

extern "C" dash_status dash_init(const dash_config *cfg, dash_model **out) {
    if (!cfg || !out) return DASH_EINVAL;
    *out = nullptr;
    dash_model *m = new dash_model();
    m->cfg = *cfg;
    const dash_config &c = m->cfg;
    dash_status st = init_check(m);
    if (st != DASH_OK) {
        delete m;
        return st;
    }
    if (c.stream) {
        m->stream = (cudaStream_t)c.stream;
        m->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete m;
            return DASH_ECUDA;
        }
        m->own_stream = true;
    }
    cudaEventCreate(&m->ev0);
    cudaEventCreate(&m->ev1);
    cudaEventCreateWithFlags(&m->ev_meta, cudaEventDisableTiming);
    for (int i = 0; i < kCopyStreams; ++i) {
        if (cudaStreamCreateWithFlags(&m->copy_streams[i], cudaStreamNonBlocking) != cudaSuccess)
            m->copy_streams[i] = nullptr;
    }
    for (int i = 0; i <= kCopyStreams; ++i) cudaEventCreateWithFlags(&m->copy_ev[i], cudaEventDisableTiming);
    for (int i = 0; i < 2; ++i) cudaEventCreateWithFlags(&m->buf_free[i], cudaEventDisableTiming);
    if (!m->copy_streams[kCopyStreams - 1]) m->copy_streams[0] = nullptr;   // all or none
    cudaGetLastError();
    st = init_alloc(m);
    if (st != DASH_OK) {
        fprintf(stderr, "dash_init: %s\n", m->err.c_str());
        free_all(m);
        if (m->own_stream) cudaStreamDestroy(m->stream);
        delete m;
        return st;
    }
    // zero the state so that get_state on an empty model is well defined
    cudaMemsetAsync(m->st.F, 0, (size_t)c.J * c.R * 8, m->stream);
    cudaMemsetAsync(m->st.G, 0, (size_t)c.R * c.R * 8, m->stream);
    *out = m;
    return DASH_OK;
}

extern "C" void dash_destroy(dash_model *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    prof_collect(m);
    if (m->err_rows) cudaFree(m->err_rows);
    if (m->err_segs) cudaFree(m->err_segs);
    if (m->re_seg_row) cudaFree(m->re_seg_row);
    if (m->re_seg_slice) cudaFree(m->re_seg_slice);
    for (cudaEvent_t e : m->prof.pool) cudaEventDestroy(e);
    for (int c = 0; c < kCopyStreams; ++c)      // split host copies still in flight
        if (m->copy_streams[c]) cudaStreamSynchronize(m->copy_streams[c]);
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    free_all(m);
    cudaEventDestroy(m->ev0);
    cudaEventDestroy(m->ev1);
    if (m->ev_meta) cudaEventDestroy(m->ev_meta);
    for (int i = 0; i < kCopyStreams; ++i)
        if (m->copy_streams[i]) cudaStreamDestroy(m->copy_streams[i]);
    for (int i = 0; i <= kCopyStreams; ++i)
        if (m->copy_ev[i]) cudaEventDestroy(m->copy_ev[i]);
    for (int i = 0; i < 2; ++i)
        if (m->buf_free[i]) cudaEventDestroy(m->buf_free[i]);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

extern "C" int64_t dash_num_slices(const dash_model *m) { return m ? m->K : -1; }

extern "C" int64_t dash_device_bytes(const dash_model *m) { return m ? m->dev_bytes : 0; }

extern "C" dash_status dash_query(const dash_model *mc, int32_t *idle) {
    if (!mc || !idle) return DASH_EINVAL;
    dash_model *m = const_cast<dash_model *>(mc);
    int32_t done = 1;
    cudaStream_t sts[1 + kCopyStreams] = {m->stream};
    for (int i = 0; i < kCopyStreams; ++i) sts[1 + i] = m->copy_streams[i];
    for (int i = 0; i <= kCopyStreams; ++i) {
        const cudaStream_t s = sts[i];
        if (i > 0 && !s) continue;                   // no copy streams on this model
        const cudaError_t e = cudaStreamQuery(s);
        if (e == cudaErrorNotReady) {
            done = 0;
        } else if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(m, DASH_ECUDA, "cudaStreamQuery: %s", cudaGetErrorString(e));
        }
    }
    *idle = done;
    return DASH_OK;
}

// After a synchronisation: an update whose bounded wait timed out was
// dropped by its own kernels (flag err[3], copied back at the end of the
// update); the host then forgets it too and reports it once.
static dash_status check_abandoned(dash_model *m) {
    if (m->h_err[3] == 0) return DASH_OK;
    m->h_err[3] = 0;
    m->K = m->K_prev;
    m->has_last = false;
    m->xx_pending = false;
    return fail(m, DASH_ETIMEOUT, "a bounded device wait timed out: the last update was dropped "
                                  "and the state is unchanged");
}

// After a synchronisation: the device counter of non-finite per-slice
// results (copied back at the end of every update) must be zero.
static dash_status check_numeric(dash_model *m) {
    if (m->h_err[4] > 0)
        return fail(m, DASH_ECUDA, "%d index self-checks of the tcgen05 kernels failed (first code %d)",
                    m->h_err[4], m->h_err[5]);
    if (dash_status a = check_abandoned(m)) return a;
    if (m->h_err[2] > 0)
        return fail(m, DASH_ENUMERIC, "%d slice factors came out non-finite", m->h_err[2]);
    return DASH_OK;
}

extern "C" dash_status dash_sync(dash_model *m) {
    if (!m) return DASH_EINVAL;
    CK(cudaStreamSynchronize(m->stream));
    return check_abandoned(m);
}

// ---------------------------------------------------------------------------
// factors / state
// ---------------------------------------------------------------------------
static dash_status refresh_gamma(dash_model *m) {
    const int J = m->cfg.J, R = m->cfg.R;
    const int64_t n = (int64_t)J * R;
    if (m->tsize == 8)
        LAUNCH(KK_CAST, k_cast<double><<<(n + 255) / 256, 256, 0, m->stream>>>(m->st.V, (double *)m->VT, n));
    else
        LAUNCH(KK_CAST, k_cast<float><<<(n + 255) / 256, 256, 0, m->stream>>>(m->st.V, (float *)m->VT, n));
    LAUNCH(KK_GAMMA, k_gamma<<<(R * R + 7) / 8, 256, 0, m->stream>>>(m->st.V, J, R, m->st.Gam, nullptr));
    if (dash_status e = launch_pinv(m, m->st.Gam, m->st.GamP, m->st.gam_ok, nullptr)) return e;
    m->gamp_fresh = true;
    m->vqr_fresh = false;
    int ok = 0;
    CK(cudaMemcpyAsync(&ok, m->st.gam_ok, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    m->gam_ok_host = ok != 0;
    m->h_fit[3] = ok;
    return DASH_OK;
}

// FP64 host array → device summaries (FP64, or double-float pairs).
static dash_status put_summ(dash_model *m, double *dst, const double *src, size_t n) {
    if (!m->df_state) {
        CK(cudaMemcpy(dst, src, n * 8, cudaMemcpyHostToDevice));
        return DASH_OK;
    }
    std::vector<float> tmp(2 * n);
    for (size_t i = 0; i < n; ++i) {
        const float hi = (float)src[i];
        tmp[2 * i] = hi;
        tmp[2 * i + 1] = (float)(src[i] - (double)hi);
    }
    CK(cudaMemcpy(dst, tmp.data(), n * 8, cudaMemcpyHostToDevice));
    return DASH_OK;
}

static dash_status get_summ(dash_model *m, double *dst, const double *src, size_t n) {
    if (!m->df_state) {
        CK(cudaMemcpy(dst, src, n * 8, cudaMemcpyDeviceToHost));
        return DASH_OK;
    }
    std::vector<float> tmp(2 * n);
    CK(cudaMemcpy(tmp.data(), src, n * 8, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) dst[i] = (double)tmp[2 * i] + (double)tmp[2 * i + 1];
    return DASH_OK;
}

static bool finite_all(const double *a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

extern "C" dash_status dash_set_factors(dash_model *m, const double *V, const double *H) {
    if (!m) return DASH_EINVAL;
    if (!V) return fail(m, DASH_EINVAL, "V is null");
    const int J = m->cfg.J, R = m->cfg.R;
    if (!finite_all(V, (size_t)J * R)) return fail(m, DASH_EINVAL, "V has non-finite entries");
    if (m->cfg.mode == DASH_MODE_Q) {
        std::vector<double> Hh((size_t)R * R, 0.0);
        if (H) {
            if (!finite_all(H, (size_t)R * R)) return fail(m, DASH_EINVAL, "H has non-finite entries");
            std::copy(H, H + (size_t)R * R, Hh.begin());
        } else {
            for (int i = 0; i < R; ++i) Hh[(size_t)i * R + i] = 1.0;
        }
        CK(cudaMemcpy(m->qH, Hh.data(), (size_t)R * R * 8, cudaMemcpyHostToDevice));
    } else if (H) {
        return fail(m, DASH_EINVAL, "H exists only in mode Q");
    }
    CK(cudaMemcpyAsync(m->st.V, V, (size_t)J * R * 8, cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    dash_status s = refresh_gamma(m);
    if (s) return s;
    m->v_set = true;
    return DASH_OK;
}

extern "C" dash_status dash_set_state_p(dash_model *m, int64_t K, const double *V,
                                        const double *W, const double *c, const double *D,
                                        const double *F, const double *G) {
    if (!m) return DASH_EINVAL;
    if (m->cfg.mode != DASH_MODE_P) return fail(m, DASH_ESTATE, "model is not in mode P");
    if (K < 0 || K > m->cfg.max_slices) return fail(m, DASH_ENOMEM, "K = %lld exceeds capacity", (long long)K);
    if (!V || !F || !G || (K > 0 && (!W || !c || !D)))
        return fail(m, DASH_EINVAL, "null state array");
    if (m->st_segs() > 0) return fail(m, DASH_ESTATE, "rows are staged; update or discard first");
    const int64_t J = m->cfg.J, R = m->cfg.R;
    CK(cudaMemcpyAsync(m->st.V, V, J * R * 8, cudaMemcpyHostToDevice, m->stream));
    if (K > 0) {
        CK(cudaMemcpyAsync(m->st.W, W, K * R * 8, cudaMemcpyHostToDevice, m->stream));
        CK(cudaStreamSynchronize(m->stream));
        dash_status s1 = put_summ(m, m->st.c, c, (size_t)K * R);
        if (s1) return s1;
        s1 = put_summ(m, m->st.D, D, (size_t)K * R * R);
        if (s1) return s1;
    }
    CK(cudaMemcpyAsync(m->st.F, F, J * R * 8, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemcpyAsync(m->st.G, G, R * R * 8, cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    m->K = K;
    dash_status s = refresh_gamma(m);
    if (s) return s;
    m->v_set = true;
    m->has_last = false;
    m->xx_valid = false;           // until dash_set_weighted_norm()
    m->xx_pending = false;
    return DASH_OK;
}

extern "C" dash_status dash_get_state_p(const dash_model *mc, double *V, double *W, double *c,
                                        double *D, double *F, double *G) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (m->cfg.mode != DASH_MODE_P) return fail(m, DASH_ESTATE, "model is not in mode P");
    CK(cudaStreamSynchronize(m->stream));
    if (dash_status a = check_numeric(m)) return a;
    const int64_t J = m->cfg.J, R = m->cfg.R, K = m->K;
    if (V) CK(cudaMemcpy(V, m->st.V, J * R * 8, cudaMemcpyDeviceToHost));
    if (W && K) CK(cudaMemcpy(W, m->st.W, K * R * 8, cudaMemcpyDeviceToHost));
    if (c && K) { dash_status s1 = get_summ(m, c, m->st.c, (size_t)K * R); if (s1) return s1; }
    if (D && K) { dash_status s1 = get_summ(m, D, m->st.D, (size_t)K * R * R); if (s1) return s1; }
    if (F) CK(cudaMemcpy(F, m->st.F, J * R * 8, cudaMemcpyDeviceToHost));
    if (G) CK(cudaMemcpy(G, m->st.G, R * R * 8, cudaMemcpyDeviceToHost));
    return DASH_OK;
}

// Mode-Q state on the host is FP64; on the device L_k, E_k and B_k^{1/2} use
// the scalar type of the R×R work (FP64, or double-float pairs) and Y_k the
// product type.  Loading a state derives E_k and B_k^{1/2} from L_k.
extern "C" dash_status dash_set_state_q(dash_model *m, int64_t K, const double *V, const double *H,
                                        const double *W, const double *L, const double *Y) {
    if (!m) return DASH_EINVAL;
    if (m->cfg.mode != DASH_MODE_Q) return fail(m, DASH_ESTATE, "model is not in mode Q");
    if (K < 0 || K > m->cfg.max_slices) return fail(m, DASH_ENOMEM, "K = %lld exceeds capacity", (long long)K);
    if (!V || !H || (K > 0 && (!W || !L || !Y))) return fail(m, DASH_EINVAL, "null state array");
    if (m->st_segs() > 0) return fail(m, DASH_ESTATE, "rows are staged; update or discard first");
    const int64_t J = m->cfg.J, R = m->cfg.R;
    if (!finite_all(V, J * R) || !finite_all(H, R * R)) return fail(m, DASH_EINVAL, "non-finite factors");
    for (int64_t k = 0; k < K; ++k)
        for (int64_t i = 0; i < R; ++i)
            for (int64_t j = 0; j < i; ++j)
                if (L[(k * R + i) * R + j] != 0.0)
                    return fail(m, DASH_EINVAL, "L_%lld is not upper-triangular", (long long)k);
    CK(cudaStreamSynchronize(m->stream));
    CK(cudaMemcpy(m->st.V, V, J * R * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->qH, H, R * R * 8, cudaMemcpyHostToDevice));
    if (K > 0) {
        CK(cudaMemcpy(m->st.W, W, K * R * 8, cudaMemcpyHostToDevice));
        dash_status s1 = put_summ(m, m->qL, L, (size_t)K * R * R);
        if (s1) return s1;
        if (m->tsize == 8) {
            CK(cudaMemcpy(m->qY, Y, (size_t)K * R * J * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> yf((size_t)K * R * J);
            for (size_t i = 0; i < yf.size(); ++i) yf[i] = (float)Y[i];
            CK(cudaMemcpy(m->qY, yf.data(), yf.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    m->K = K;
    dash_status s = refresh_gamma(m);
    if (s) return s;
    s = prepare_q(m);
    if (s) return s;
    CK(cudaStreamSynchronize(m->stream));
    m->v_set = true;
    m->has_last = false;
    return DASH_OK;
}

// Fold the last finished update's ||X_new||² (h_fit[1]) into xx.  Call only
// after the model's stream has been synchronised.
static void fold_xx(dash_model *m) {
    if (!m->xx_pending) return;
    m->xx = m->xx_lam * m->xx + m->h_fit[1];
    m->xx_pending = false;
}

extern "C" dash_status dash_get_state_q(const dash_model *mc, double *V, double *H, double *W,
                                        double *L, double *Y) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (m->cfg.mode != DASH_MODE_Q) return fail(m, DASH_ESTATE, "model is not in mode Q");
    const int64_t J = m->cfg.J, R = m->cfg.R, K = m->K;
    CK(cudaStreamSynchronize(m->stream));
    if (dash_status sn = check_numeric(m)) return sn;
    if (V) CK(cudaMemcpy(V, m->st.V, J * R * 8, cudaMemcpyDeviceToHost));
    if (H) CK(cudaMemcpy(H, m->qH, R * R * 8, cudaMemcpyDeviceToHost));
    if (W && K) CK(cudaMemcpy(W, m->st.W, K * R * 8, cudaMemcpyDeviceToHost));
    if (L && K) { dash_status s1 = get_summ(m, L, m->qL, (size_t)K * R * R); if (s1) return s1; }
    if (Y && K) {
        if (m->tsize == 8) {
            CK(cudaMemcpy(Y, m->qY, (size_t)K * R * J * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> yf((size_t)K * R * J);
            CK(cudaMemcpy(yf.data(), m->qY, yf.size() * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < yf.size(); ++i) Y[i] = yf[i];
        }
    }
    return DASH_OK;
}

extern "C" dash_status dash_factors(const dash_model *mc, double *V, double *W, int64_t k_first,
                                    int64_t k_count, double *H) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    const int64_t J = m->cfg.J, R = m->cfg.R;
    if (W && (k_first < 0 || k_count < 0 || k_first + k_count > m->K))
        return fail(m, DASH_EINVAL, "slice range %lld+%lld outside 0..%lld", (long long)k_first,
                    (long long)k_count, (long long)m->K);
    CK(cudaStreamSynchronize(m->stream));
    if (V) CK(cudaMemcpy(V, m->st.V, J * R * 8, cudaMemcpyDeviceToHost));
    if (W && k_count)
        CK(cudaMemcpy(W, m->st.W + k_first * R, k_count * R * 8, cudaMemcpyDeviceToHost));
    if (H) {
        if (m->cfg.mode != DASH_MODE_Q) return fail(m, DASH_ESTATE, "H exists only in mode Q");
        CK(cudaMemcpy(H, m->qH, R * R * 8, cudaMemcpyDeviceToHost));
    }
    return DASH_OK;
}

extern "C" dash_status dash_new_rows(const dash_model *mc, double *out, int64_t *n_rows) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (n_rows) *n_rows = m->has_last ? m->last_N : 0;
    if (!m->has_last || !out) return DASH_OK;
    const int64_t n = m->last_N * m->cfg.R;
    CK(cudaStreamSynchronize(m->stream));
    if (m->tsize == 8) {
        CK(cudaMemcpy(out, m->U, n * 8, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp(n);
        CK(cudaMemcpy(tmp.data(), m->U, n * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) out[i] = tmp[i];
    }
    return DASH_OK;
}

extern "C" dash_status dash_fitness(const dash_model *mc, double *fit_batch, double *x_norm2) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (!m->has_last) return fail(m, DASH_ESTATE, "no update has run");
    CK(cudaStreamSynchronize(m->stream));
    if (dash_status sn = check_numeric(m)) return sn;
    if (fit_batch) *fit_batch = m->h_fit[0];
    if (x_norm2) *x_norm2 = m->h_fit[1];
    return DASH_OK;
}

extern "C" dash_status dash_fitness_lambda(const dash_model *mc, double *fit_lambda, double *x_norm2_lambda) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (m->cfg.mode != DASH_MODE_P) return fail(m, DASH_ESTATE, "the lambda-weighted fitness is defined in mode P");
    CK(cudaStreamSynchronize(m->stream));
    if (dash_status sn = check_numeric(m)) return sn;
    fold_xx(m);
    if (!m->xx_valid)
        return fail(m, DASH_ESTATE, "the weighted norm of the absorbed rows is unknown (dash_set_weighted_norm)");
    const int J = m->cfg.J, R = m->cfg.R;
    LAUNCH(KK_FIT_LAMBDA, k_fit_lambda<<<1, 32, 0, m->stream>>>(m->st.V, m->st.F, m->st.Gam, m->st.G, J, R, m->xx,
                                                                m->fit + 4));
    double out[2];
    CK(cudaMemcpyAsync(out, m->fit + 4, 2 * 8, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (fit_lambda) *fit_lambda = out[0];
    if (x_norm2_lambda) *x_norm2_lambda = m->xx;
    return DASH_OK;
}

extern "C" dash_status dash_set_weighted_norm(dash_model *m, double x_norm2_lambda) {
    if (!m) return DASH_EINVAL;
    if (!(x_norm2_lambda >= 0.0) || !std::isfinite(x_norm2_lambda))
        return fail(m, DASH_EINVAL, "the weighted norm must be finite and >= 0");
    CK(cudaStreamSynchronize(m->stream));
    fold_xx(m);
    m->xx = x_norm2_lambda;
    m->xx_valid = true;
    return DASH_OK;
}

extern "C" dash_status dash_last_plan(const dash_model *mc, int64_t *tile_rows,
                                      int64_t *tile_slices, int64_t *tiles, int64_t *chunk_rows,
                                      int64_t *general_rows) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (!m->has_last) return fail(m, DASH_ESTATE, "no update has run");
    if (tile_rows) *tile_rows = m->plan_tile_rows;
    if (tile_slices) *tile_slices = m->plan_tile_slices;
    if (tiles) *tiles = m->plan_tiles;
    if (chunk_rows) *chunk_rows = m->plan_chunk_rows;
    if (general_rows) *general_rows = m->plan_general_rows;
    return DASH_OK;
}

extern "C" dash_status dash_set_wait_limit(dash_model *m, int64_t cycles) {
    if (!m) return DASH_EINVAL;
    if (cycles < 1000) return fail(m, DASH_EINVAL, "wait limit below 1000 cycles");
    m->wait_limit = cycles;
    return DASH_OK;
}

extern "C" dash_status dash_inject_wait_fault(dash_model *m) {
    if (!m) return DASH_EINVAL;
    if (m->cfg.mode != DASH_MODE_P || m->xu_nst == 0)
        return fail(m, DASH_ESTATE, "no tcgen05 X·Q_V pass in this configuration");
    m->inject_wait_fault = 1;
    return DASH_OK;
}

extern "C" dash_status dash_set_graph(dash_model *m, int32_t on) {
    if (!m) return DASH_EINVAL;
    if (on != 0 && on != 1) return fail(m, DASH_EINVAL, "graph switch must be 0 or 1");
    CK(cudaStreamSynchronize(m->stream));
    m->use_graph = on != 0;
    if (!m->use_graph && m->gexec) {
        cudaGraphExecDestroy(m->gexec);
        m->gexec = nullptr;
    }
    return DASH_OK;
}

extern "C" dash_status dash_set_autotune(dash_model *m, int32_t on) {
    if (!m) return DASH_EINVAL;
    if (on != 0 && on != 1) return fail(m, DASH_EINVAL, "autotune switch must be 0 or 1");
    m->autotune = on != 0;
    return DASH_OK;
}

extern "C" dash_status dash_autotune_result(const dash_model *m, int32_t *n_candidates, int32_t *chosen,
                                            int32_t *resident, int32_t *ring, float *ms) {
    if (!m) return DASH_EINVAL;
    if (n_candidates) *n_candidates = m->xu_tuned ? m->xu_tune_n : 0;
    if (chosen) *chosen = m->xu_tuned ? m->xu_tune_best : -1;
    if (resident) *resident = m->xr_nst > 0 ? 1 : 0;
    if (ring) *ring = m->xr_nst > 0 ? m->xr_nst : m->xu_nst;
    if (ms)
        for (int i = 0; i < 8; ++i) ms[i] = (m->xu_tuned && i < m->xu_tune_n) ? m->xu_tune_ms[i] : 0.f;
    return DASH_OK;
}

extern "C" dash_status dash_graph_stats(const dash_model *m, int64_t *instantiations, int64_t *updates) {
    if (!m) return DASH_EINVAL;
    if (instantiations) *instantiations = m->graph_instantiations;
    if (updates) *updates = m->graph_updates;
    return DASH_OK;
}

extern "C" dash_status dash_set_row_path(dash_model *m, int32_t path) {
    if (!m) return DASH_EINVAL;
    if (path != DASH_ROWS_AUTO && path != DASH_ROWS_FUSED && path != DASH_ROWS_SPLIT &&
        path != DASH_ROWS_SPLIT_WARP)
        return fail(m, DASH_EINVAL, "unknown row path %d", path);
    m->row_path = path;
    return DASH_OK;
}

// ---------------------------------------------------------------------------
// reconstruction errors of the last update (Definitions 1-2)
// ---------------------------------------------------------------------------
template <typename TI, typename T>
static dash_status launch_resid(dash_model *m, int64_t N, int n_seg) {
    const int J = m->cfg.J, R = m->cfg.R;
    const size_t smem = err_smem<T>(R, J);
    CK(cudaFuncSetAttribute(k_resid_rows<TI, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>((N + 7) / 8, 4 * (int64_t)m->n_sm);
    LAUNCH(KK_Q_OUT, (k_resid_rows<TI, T><<<grid, 256, smem, m->stream>>>(
                         N, J, R, n_seg, m->d_seg_row, m->d_seg_slice, (const TI *)m->last_X,
                         (const T *)m->U, m->cfg.mode == DASH_MODE_Q ? m->qH : nullptr, m->st.W,
                         (const T *)m->VT, m->err_rows)));
    return DASH_OK;
}

extern "C" dash_status dash_local_errors(dash_model *m, double *te, double *fit_direct, double *se,
                                         int64_t se_len) {
    if (!m) return DASH_EINVAL;
    if (!m->has_last) return fail(m, DASH_ESTATE, "no update has run");
    if (!m->last_X && m->last_N > 0)
        return fail(m, DASH_ESTATE, "the last batch's rows are gone (rows were staged since)");
    if (se && se_len < m->K) return fail(m, DASH_EINVAL, "se needs %lld entries", (long long)m->K);
    const int64_t N = m->last_N;
    const int n_seg = (int)m->last_ids.size();
    const int J = m->cfg.J;
    if (N > 0) {
        if (m->err_rows_cap < N) {
            if (m->err_rows) cudaFree(m->err_rows);
            m->err_rows = nullptr;
            CK(cudaMalloc(&m->err_rows, (size_t)N * 3 * 8));
            m->err_rows_cap = N;
        }
        if (m->err_segs_cap < n_seg) {
            if (m->err_segs) cudaFree(m->err_segs);
            m->err_segs = nullptr;
            CK(cudaMalloc(&m->err_segs, (size_t)n_seg * 3 * 8));
            m->err_segs_cap = n_seg;
        }
        const bool f64in = m->cfg.input_dtype == DASH_F64;
        dash_status s;
        if (m->tsize == 8) s = f64in ? launch_resid<double, double>(m, N, n_seg) : launch_resid<float, double>(m, N, n_seg);
        else s = f64in ? launch_resid<double, float>(m, N, n_seg) : launch_resid<float, float>(m, N, n_seg);
        if (s) return s;
        LAUNCH(KK_Q_FIT, (k_resid_segs<<<(n_seg + 127) / 128, 128, 0, m->stream>>>(n_seg, m->d_seg_row,
                                                                                 m->err_rows, m->err_segs)));
    }
    std::vector<double> seg((size_t)n_seg * 3, 0.0);
    if (N > 0) CK(cudaMemcpyAsync(seg.data(), m->err_segs, seg.size() * 8, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    // group segments by slice, in segment order; te averages over the slices
    // with new rows, in ascending slice order
    std::vector<double> abs_k(m->K, 0.0);
    std::vector<int64_t> n_k(m->K, 0);
    double sq = 0.0, xn = 0.0;
    for (int s = 0; s < n_seg; ++s) {
        const int64_t k = m->last_ids[s];
        abs_k[k] += seg[(size_t)s * 3];
        n_k[k] += m->last_rp[s + 1] - m->last_rp[s];
        sq += seg[(size_t)s * 3 + 1];
        xn += seg[(size_t)s * 3 + 2];
    }
    double tsum = 0.0;
    int64_t tcount = 0;
    for (int64_t k = 0; k < m->K; ++k) {
        const double v = n_k[k] > 0 ? abs_k[k] / ((double)n_k[k] * J) : NAN;
        if (n_k[k] > 0) {
            tsum += v;
            ++tcount;
        }
        if (se) se[k] = v;
    }
    if (te) *te = tcount ? tsum / (double)tcount : 0.0;
    if (fit_direct) *fit_direct = xn > 0.0 ? 1.0 - std::sqrt(sq / xn) : 1.0;
    return DASH_OK;
}

// Reconstruction error of arbitrary rows (the global error over an
// accumulated tensor) against the current factors.
template <typename TI>
static dash_status launch_rows_error(dash_model *m, int64_t N, int n_seg, const void *X,
                                     const double *rows) {
    const int J = m->cfg.J, R = m->cfg.R;
    const size_t smem = err_smem<double>(R, J);
    CK(cudaFuncSetAttribute(k_resid_rows<TI, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>((N + 7) / 8, 4 * (int64_t)m->n_sm);
    LAUNCH(KK_Q_OUT, (k_resid_rows<TI, double><<<grid, 256, smem, m->stream>>>(
                         N, J, R, n_seg, m->re_seg_row, m->re_seg_slice, (const TI *)X, rows,
                         m->cfg.mode == DASH_MODE_Q ? m->qH : nullptr, m->st.W, m->st.V,
                         m->err_rows)));
    return DASH_OK;
}

extern "C" dash_status dash_rows_error(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                                       const int64_t *row_ptr, const void *X, const double *rows,
                                       double *sq_err, double *sq_x, double *abs_err) {
    if (!m) return DASH_EINVAL;
    if (m->broken) return fail(m, DASH_ESTATE, "model is unusable after a CUDA error");
    if (n_seg < 0 || (n_seg > 0 && (!slice_ids || !row_ptr)))
        return fail(m, DASH_EINVAL, "bad segment arrays");
    if (n_seg > INT32_MAX) return fail(m, DASH_EINVAL, "too many segments");
    if (n_seg > 0 && row_ptr[0] != 0) return fail(m, DASH_EINVAL, "row_ptr[0] must be 0");
    for (int64_t q = 0; q < n_seg; ++q) {
        if (row_ptr[q + 1] < row_ptr[q]) return fail(m, DASH_EINVAL, "row_ptr is not ascending");
        if (slice_ids[q] < 0 || slice_ids[q] >= m->K)
            return fail(m, DASH_EINVAL, "slice id %lld is not in the model", (long long)slice_ids[q]);
    }
    const int64_t N = n_seg ? row_ptr[n_seg] : 0;
    if (N > 0 && (!X || !rows)) return fail(m, DASH_EINVAL, "X or rows is null");
    double e2 = 0.0, x2 = 0.0, ea = 0.0;
    if (N > 0) {
        if (m->err_rows_cap < N) {
            if (m->err_rows) cudaFree(m->err_rows);
            m->err_rows = nullptr;
            CK(cudaMalloc(&m->err_rows, (size_t)N * 3 * 8));
            m->err_rows_cap = N;
        }
        if (m->err_segs_cap < n_seg) {
            if (m->err_segs) cudaFree(m->err_segs);
            m->err_segs = nullptr;
            CK(cudaMalloc(&m->err_segs, (size_t)n_seg * 3 * 8));
            m->err_segs_cap = n_seg;
        }
        if (m->re_cap < n_seg) {
            if (m->re_seg_row) cudaFree(m->re_seg_row);
            if (m->re_seg_slice) cudaFree(m->re_seg_slice);
            m->re_seg_row = nullptr;
            m->re_seg_slice = nullptr;
            CK(cudaMalloc(&m->re_seg_row, (size_t)(n_seg + 1) * 8));
            CK(cudaMalloc(&m->re_seg_slice, (size_t)n_seg * 4));
            m->re_cap = n_seg;
        }
        std::vector<int> ids32(slice_ids, slice_ids + n_seg);
        CK(cudaMemcpyAsync(m->re_seg_row, row_ptr, (size_t)(n_seg + 1) * 8, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->re_seg_slice, ids32.data(), (size_t)n_seg * 4, cudaMemcpyHostToDevice, m->stream));
        const dash_status st = m->cfg.input_dtype == DASH_F64
                                   ? launch_rows_error<double>(m, N, (int)n_seg, X, rows)
                                   : launch_rows_error<float>(m, N, (int)n_seg, X, rows);
        if (st) return st;
        LAUNCH(KK_Q_FIT, (k_resid_segs<<<(unsigned)((n_seg + 127) / 128), 128, 0, m->stream>>>(
                             (int)n_seg, m->re_seg_row, m->err_rows, m->err_segs)));
        std::vector<double> seg((size_t)n_seg * 3);
        CK(cudaMemcpyAsync(seg.data(), m->err_segs, seg.size() * 8, cudaMemcpyDeviceToHost, m->stream));
        CK(cudaStreamSynchronize(m->stream));    // also keeps ids32 alive for its copy
        for (int64_t q = 0; q < n_seg; ++q) {
            ea += seg[(size_t)q * 3];
            e2 += seg[(size_t)q * 3 + 1];
            x2 += seg[(size_t)q * 3 + 2];
        }
    }
    if (sq_err) *sq_err = e2;
    if (sq_x) *sq_x = x2;
    if (abs_err) *abs_err = ea;
    return DASH_OK;
}

extern "C" dash_status dash_last_update_ms(const dash_model *mc, float *ms) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m || !ms) return DASH_EINVAL;
    if (!m->has_last) return fail(m, DASH_ESTATE, "no update has run");
    CK(cudaEventSynchronize(m->ev1));
    CK(cudaEventElapsedTime(ms, m->ev0, m->ev1));
    return DASH_OK;
}

// ---------------------------------------------------------------------------
// staging
// ---------------------------------------------------------------------------
static dash_status stage_rows(dash_model *m, int64_t k, const void *X, int64_t I, int64_t ld,
                              int32_t where) {
    m->last_X = nullptr;                  // the staging buffer is about to be reused
    const int64_t J = m->cfg.J;
    const size_t ie = (m->cfg.input_dtype == DASH_F64) ? 8 : 4;
    if (I < 0) return fail(m, DASH_EINVAL, "negative row count");
    if (I > 0 && !X) return fail(m, DASH_EINVAL, "X is null");
    if (ld < J) return fail(m, DASH_EINVAL, "ld %lld < J %lld", (long long)ld, (long long)J);
    if (where != DASH_HOST && where != DASH_DEVICE) return fail(m, DASH_EINVAL, "bad pointer location");
    if (m->st_rows + I > m->stage_cap)
        return fail(m, DASH_ENOMEM, "staged rows would exceed the staging capacity %lld", (long long)m->stage_cap);
    if (m->st_segs() + 1 > m->cfg.max_segments)
        return fail(m, DASH_ENOMEM, "staged segments would exceed max_segments");
    if (I > 0) {
        char *dst = (char *)m->Xs + (size_t)m->st_rows * J * ie;
        CK(cudaMemcpy2DAsync(dst, J * ie, X, ld * ie, J * ie, I,
                             where == DASH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                             m->stream));
    }
    m->st_slice.push_back(k);
    m->st_rows += I;
    m->st_row.push_back(m->st_rows);
    return DASH_OK;
}

extern "C" dash_status dash_append_rows(dash_model *m, int64_t k, const void *X, int64_t I_new,
                                        int64_t ld, int32_t where) {
    if (!m) return DASH_EINVAL;
    if (k < 0 || k >= m->K + m->st_new)
        return fail(m, DASH_EINVAL, "slice %lld does not exist (K = %lld, staged new = %lld)",
                    (long long)k, (long long)m->K, (long long)m->st_new);
    return stage_rows(m, k, X, I_new, ld, where);
}

extern "C" dash_status dash_append_slices(dash_model *m, int64_t L, const int64_t *I,
                                          const void *const *X, const int64_t *ld, int32_t where,
                                          int64_t *first_new_id) {
    if (!m) return DASH_EINVAL;
    if (L < 0 || (L > 0 && (!I || !X))) return fail(m, DASH_EINVAL, "bad slice list");
    if (m->K + m->st_new + L > m->cfg.max_slices)
        return fail(m, DASH_ENOMEM, "slices would exceed max_slices = %lld", (long long)m->cfg.max_slices);
    int64_t tot = 0;
    for (int64_t l = 0; l < L; ++l) {
        if (I[l] < 0) return fail(m, DASH_EINVAL, "negative row count for new slice %lld", (long long)l);
        tot += I[l];
    }
    if (m->st_rows + tot > m->stage_cap) return fail(m, DASH_ENOMEM, "staged rows would exceed the staging capacity");
    if (m->st_segs() + L > m->cfg.max_segments) return fail(m, DASH_ENOMEM, "staged segments would exceed max_segments");
    if (first_new_id) *first_new_id = m->K + m->st_new;
    for (int64_t l = 0; l < L; ++l) {
        const int64_t id = m->K + m->st_new;
        m->st_new += 1;
        dash_status s = stage_rows(m, id, X[l], I[l], ld ? ld[l] : m->cfg.J, where);
        if (s) return s;
    }
    return DASH_OK;
}

// Check a CSR batch: ascending row_ptr from 0, ids in range, new ids
// consecutive from K_base.  Returns the number of new slices in *n_new.
static dash_status check_csr(dash_model *m, int64_t n_seg, const int64_t *ids, const int64_t *rp,
                             int64_t K_base, int64_t *n_new) {
    if (n_seg < 0 || (n_seg > 0 && (!ids || !rp))) return fail(m, DASH_EINVAL, "bad CSR arrays");
    if (n_seg > 0 && rp[0] != 0) return fail(m, DASH_EINVAL, "row_ptr[0] must be 0");
    int64_t next_new = K_base;
    for (int64_t s = 0; s < n_seg; ++s) {
        if (rp[s + 1] < rp[s]) return fail(m, DASH_EINVAL, "row_ptr not ascending at %lld", (long long)s);
        const int64_t k = ids[s];
        if (k < 0) return fail(m, DASH_EINVAL, "negative slice id");
        if (k >= K_base) {
            if (k == next_new) ++next_new;
            else if (k >= next_new)
                return fail(m, DASH_EINVAL, "new slice ids must be consecutive from %lld (got %lld)",
                            (long long)K_base, (long long)k);
        }
    }
    *n_new = next_new - K_base;
    return DASH_OK;
}

extern "C" dash_status dash_append_batch(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                                         const int64_t *row_ptr, const void *X, int32_t where) {
    if (!m) return DASH_EINVAL;
    m->last_X = nullptr;                  // the staging buffer is about to be reused
    int64_t n_new = 0;
    dash_status s = check_csr(m, n_seg, slice_ids, row_ptr, m->K + m->st_new, &n_new);
    if (s) return s;
    const int64_t N = n_seg ? row_ptr[n_seg] : 0;
    if (m->st_rows + N > m->stage_cap) return fail(m, DASH_ENOMEM, "staged rows would exceed the staging capacity");
    if (m->st_segs() + n_seg > m->cfg.max_segments) return fail(m, DASH_ENOMEM, "staged segments would exceed max_segments");
    if (m->K + m->st_new + n_new > m->cfg.max_slices) return fail(m, DASH_ENOMEM, "slices would exceed max_slices");
    if (N > 0 && !X) return fail(m, DASH_EINVAL, "X is null");
    const size_t ie = (m->cfg.input_dtype == DASH_F64) ? 8 : 4;
    if (N > 0) {
        char *dst = (char *)m->Xs + (size_t)m->st_rows * m->cfg.J * ie;
        const size_t bytes = (size_t)N * m->cfg.J * ie;
        if (where == DASH_HOST && bytes >= kSplitCopyBytes && m->copy_streams[0]) {
            // a large host batch: one copy per part on the copy streams, so
            // several copy engines share it.  The parts wait only until the
            // last update that read this staging buffer is done, so they
            // overlap an update in flight on the other buffer; the next
            // update makes the model's stream wait for them.
            const size_t part = (bytes / kCopyStreams + 4095) / 4096 * 4096;
            for (int i = 0; i < kCopyStreams; ++i) {
                const size_t off = (size_t)i * part;
                const size_t nb = off >= bytes ? 0 : (bytes - off < part ? bytes - off : part);
                CK(cudaStreamWaitEvent(m->copy_streams[i], m->buf_free[m->st_buf], 0));
                if (nb > 0)
                    CK(cudaMemcpyAsync(dst + off, (const char *)X + off, nb, cudaMemcpyHostToDevice,
                                       m->copy_streams[i]));
                CK(cudaEventRecord(m->copy_ev[i], m->copy_streams[i]));
            }
            m->copies_pending = true;
        } else {
            CK(cudaMemcpyAsync(dst, X, bytes,
                               where == DASH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                               m->stream));
        }
    }
    const int64_t base = m->st_rows;
    for (int64_t q = 0; q < n_seg; ++q) {
        m->st_slice.push_back(slice_ids[q]);
        m->st_row.push_back(base + row_ptr[q + 1]);
    }
    m->st_rows += N;
    m->st_new += n_new;
    return DASH_OK;
}

// ---------------------------------------------------------------------------
// one update
// ---------------------------------------------------------------------------

// Build and upload the device view of a batch: segments, touched slices and
// their segment lists, tiles for the fused row kernel (slices with one segment
// of at most FU_TILE_MAX rows) and the runs of rows left to the general
// kernels.  K_old is the slice count before the update.
static dash_status plan_batch(dash_model *m, int64_t n_seg, const int64_t *ids,
                              const int64_t *rp /* n_seg+1 absolute */, int64_t K_old,
                              int64_t n_new, const void *X, bool allow_fused, BatchDev *b) {
    const int64_t K_all = K_old + n_new;
    // The pinned metadata buffers are rewritten below: wait until the last
    // batch's copies out of them have run (they open that update, so this
    // seldom waits).  The host planning then overlaps the previous update on
    // the GPU.  It assumes the last known state of Γ (nonsingular or not) and
    // is redone in the rare case that the previous update changed it.
    m->prof.t_plan0 = std::chrono::steady_clock::now();
    CK(cudaEventSynchronize(m->ev_meta));
    bool gam_ok = m->gam_ok_host;
    int n_touch = 0, nt = 0, nr = 0;
    int64_t ng = 0;
    for (int pass = 0;; ++pass) {
    int *tslot = m->h_tslot;
    for (int64_t k = 0; k < K_all; ++k) tslot[k] = -1;
    std::vector<int> cnt;
    cnt.reserve(1024);
    n_touch = 0;
    for (int64_t s = 0; s < n_seg; ++s) {
        const int64_t k = ids[s];
        if (tslot[k] < 0) {
            tslot[k] = n_touch++;
            cnt.push_back(0);
        }
        cnt[tslot[k]] += 1;
    }
    // which segments the fused kernel finishes
    const bool fused = allow_fused && m->fused_ok && gam_ok && ((uintptr_t)X % 16) == 0;
    // split: no tiles, every touched slice through the chunked path
    const bool split = fused && m->cfg.precision == DASH_PREC_F16X3 &&
                       (m->row_path == DASH_ROWS_SPLIT || m->row_path == DASH_ROWS_SPLIT_WARP ||
                        (m->row_path == DASH_ROWS_AUTO && kAutoSplit));
    m->split_active = split;
    std::vector<char> fz(n_seg, 0);
    if (fused && !split) {
        for (int64_t s = 0; s < n_seg; ++s)
            fz[s] = cnt[tslot[ids[s]]] == 1 && rp[s + 1] - rp[s] <= FU_TILE_MAX;
    }
    m->fused_active = fused;
    // renumber touched slots in ascending slice order (fixed reduction order);
    // slices finished by the fused kernel get -2
    {
        int t = 0;
        std::vector<int> remap(n_touch, -1), fused_slot(n_touch, 0);
        for (int64_t s = 0; s < n_seg; ++s)
            if (fz[s]) fused_slot[tslot[ids[s]]] = 1;
        std::vector<int> c2;
        c2.reserve(n_touch);
        for (int64_t k = 0; k < K_all; ++k) {
            if (tslot[k] < 0) continue;
            const int old = tslot[k];
            if (fused_slot[old]) {
                tslot[k] = -2;
            } else {
                remap[old] = t;
                tslot[k] = t++;
                c2.push_back(cnt[old]);
            }
        }
        cnt.swap(c2);
        n_touch = t;
    }
    int *tp = m->h_tseg_ptr;
    tp[0] = 0;
    for (int i = 0; i < n_touch; ++i) tp[i + 1] = tp[i] + cnt[i];
    std::vector<int> fillp(tp, tp + n_touch);
    for (int64_t s = 0; s < n_seg; ++s) {
        const int t = tslot[ids[s]];
        if (t >= 0) m->h_tseg_idx[fillp[t]++] = (int)s;
        m->h_seg_slice[s] = (int)ids[s];
    }
    // fused path: the remaining touched slices are split into chunks, and
    // every slice not finished by a tile (chunked or untouched) gets a finish entry
    m->n_chunks = 0;
    m->n_fin = 0;
    if (fused) {
        int nc = 0, nf = 0;
        for (int64_t k = 0; k < K_all; ++k) {
            const int t = tslot[k];
            if (t < 0) continue;
            m->h_fin_k[nf] = (int)k;
            m->h_fin_c0[nf] = nc;
            ++nf;
            for (int q = tp[t]; q < tp[t + 1]; ++q) {
                const int sg = m->h_tseg_idx[q];
                for (int64_t r = rp[sg]; r < rp[sg + 1]; r += FU_TILE_MAX) {
                    m->h_ch_row0[nc] = r;
                    m->h_ch_n[nc] = (int)std::min<int64_t>(FU_TILE_MAX, rp[sg + 1] - r);
                    m->h_ch_k[nc] = (int)k;
                    ++nc;
                }
            }
        }
        for (int64_t k = 0; k < K_all; ++k) {
            if (tslot[k] != -1) continue;
            m->h_fin_k[nf] = (int)k;
            m->h_fin_c0[nf] = nc;
            ++nf;
        }
        m->h_fin_c0[nf] = nc;
        m->n_chunks = nc;
        m->n_fin = nf;
    }
    for (int64_t s = 0; s <= n_seg; ++s) m->h_seg_row[s] = rp[s];
    // tiles: runs of consecutive fused segments with <= FU_TILE_MAX rows
    nt = 0;
    {
        int64_t s = 0;
        while (s < n_seg) {
            if (!fz[s]) { ++s; continue; }
            const int64_t s0 = s;
            int64_t rows = 0;
            while (s < n_seg && fz[s] && rows + (rp[s + 1] - rp[s]) <= FU_TILE_MAX) {
                rows += rp[s + 1] - rp[s];
                ++s;
            }
            m->h_tile_s0[nt] = (int)s0;
            m->h_tile_s1[nt] = (int)s;
            ++nt;
        }
    }
    m->n_tiles = nt;
    {
        int64_t tr = 0, ts = 0;
        for (int64_t q = 0; q < n_seg; ++q)
            if (fz[q]) {
                tr += rp[q + 1] - rp[q];
                ++ts;
            }
        m->plan_tile_rows = tr;
        m->plan_tile_slices = ts;
        m->plan_tiles = nt;
    }
    // general runs: maximal runs of consecutive non-fused segments
    nr = 0;
    ng = 0;
    {
        int64_t s = 0;
        while (s < n_seg) {
            if (fz[s]) { ++s; continue; }
            const int64_t s0 = s;
            while (s < n_seg && !fz[s]) ++s;
            const int64_t rows = rp[s] - rp[s0];
            if (rows > 0) {
                m->h_run_row0[nr] = rp[s0];
                m->h_run_g0[nr] = ng;
                ++nr;
                ng += rows;
            }
        }
        m->h_run_g0[nr] = ng;
    }
    // with the fused path on, the rows outside tiles go through the chunked path
    m->plan_chunk_rows = fused ? ng : 0;
    m->plan_general_rows = fused ? 0 : ng;
    if (pass == 0) {
        const auto th0 = std::chrono::steady_clock::now();
        CK(cudaStreamSynchronize(m->stream));   // the previous update has finished
        fold_xx(m);
        if (m->prof.on) {
            const auto th1 = std::chrono::steady_clock::now();
            m->prof.ms[KK_HOST_PLAN] += std::chrono::duration<double, std::milli>(th0 - m->prof.t_plan0).count();
            m->prof.ms[KK_HOST_WAIT] += std::chrono::duration<double, std::milli>(th1 - th0).count();
            m->prof.launches[KK_HOST_PLAN] += 1;
            m->prof.launches[KK_HOST_WAIT] += 1;
        }
        m->gam_ok_host = m->h_fit[3] != 0.0;
        if (dash_status a = check_abandoned(m)) return a;
        if (m->h_err[2] > 0)
            return fail(m, DASH_ENUMERIC, "%d slice factors came out non-finite", m->h_err[2]);
        if (m->gam_ok_host != gam_ok) {
            gam_ok = m->gam_ok_host;
            continue;
        }
    }
    break;
    }
    if (m->n_chunks > 0) {
        const int nc = m->n_chunks;
        CK(cudaMemcpyAsync(m->d_ch_row0, m->h_ch_row0, nc * 8, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->d_ch_n, m->h_ch_n, nc * 4, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->d_ch_k, m->h_ch_k, nc * 4, cudaMemcpyHostToDevice, m->stream));
    }
    if (m->fused_active) {
        const int nf = m->n_fin;
        if (nf > 0) CK(cudaMemcpyAsync(m->d_fin_k, m->h_fin_k, nf * 4, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->d_fin_c0, m->h_fin_c0, (nf + 1) * 4, cudaMemcpyHostToDevice, m->stream));
    }
    if (n_seg > 0) {
        CK(cudaMemcpyAsync(m->d_seg_slice, m->h_seg_slice, n_seg * 4, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->d_tseg_idx, m->h_tseg_idx, n_seg * 4, cudaMemcpyHostToDevice, m->stream));
    }
    CK(cudaMemcpyAsync(m->d_seg_row, m->h_seg_row, (n_seg + 1) * 8, cudaMemcpyHostToDevice, m->stream));
    CK(cudaMemcpyAsync(m->d_tseg_ptr, m->h_tseg_ptr, (n_touch + 1) * 4, cudaMemcpyHostToDevice, m->stream));
    if (K_all > 0) CK(cudaMemcpyAsync(m->d_tslot, m->h_tslot, K_all * 4, cudaMemcpyHostToDevice, m->stream));
    if (nt > 0) {
        CK(cudaMemcpyAsync(m->d_tile_s0, m->h_tile_s0, nt * 4, cudaMemcpyHostToDevice, m->stream));
        CK(cudaMemcpyAsync(m->d_tile_s1, m->h_tile_s1, nt * 4, cudaMemcpyHostToDevice, m->stream));
    }
    CK(cudaMemcpyAsync(m->d_run_g0, m->h_run_g0, (nr + 1) * 8, cudaMemcpyHostToDevice, m->stream));
    if (nr > 0) CK(cudaMemcpyAsync(m->d_run_row0, m->h_run_row0, nr * 8, cudaMemcpyHostToDevice, m->stream));
    CK(cudaEventRecord(m->ev_meta, m->stream));
    const int64_t N = n_seg ? rp[n_seg] : 0;
    b->n_seg = (int)n_seg;
    b->n_touch = n_touch;
    b->K_all = (int)K_all;
    b->K_old = (int)K_old;
    b->N = N;
    b->seg_slice = m->d_seg_slice;
    b->seg_row = m->d_seg_row;
    b->tslot = m->d_tslot;
    b->tseg_ptr = m->d_tseg_ptr;
    b->tseg_idx = m->d_tseg_idx;
    b->row_slice = m->d_row_slice;
    b->n_runs = nr;
    b->N_gen = ng;
    b->run_g0 = m->d_run_g0;
    b->run_row0 = m->d_run_row0;
    return DASH_OK;
}

static dash_status run_update(dash_model *m, const BatchDev &b, const void *X, double lam,
                              bool begin_new) {
    if (m->cfg.mode == DASH_MODE_Q) return run_update_q(m, b, X, lam, begin_new, true);
    return run_update_p(m, b, X, lam, begin_new);
}

// The kernels of one update: Algorithm 1 once, or n_sweeps times over the
// same new rows with the old helpers restored before every further pass.
static dash_status launch_sweeps(dash_model *m, const BatchDev &b, const void *X) {
    dash_status s;
    const int nsw = m->cfg.mode == DASH_MODE_P ? m->cfg.n_sweeps : 1;
    if (nsw > 1) {
        // the old helpers every pass starts from (new slices start at zero)
        const int64_t R = m->cfg.R;
        CK(cudaMemcpyAsync(m->sw_c, m->st.c, m->K * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->sw_D, m->st.D, m->K * R * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->sw_F, m->st.F, (size_t)m->cfg.J * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->sw_G, m->st.G, R * R * 8, cudaMemcpyDeviceToDevice, m->stream));
    }
    s = run_update(m, b, X, m->cfg.lambda, true);
    if (s) return s;
    for (int sw = 1; sw < nsw; ++sw) {
        // Algorithm 1 again on the same rows with the factors of the last
        // pass and the old helpers held fixed
        const int64_t R = m->cfg.R, Ka = b.K_all;
        CK(cudaMemcpyAsync(m->st.c, m->sw_c, m->K * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->st.D, m->sw_D, m->K * R * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        if (Ka > m->K) {
            CK(cudaMemsetAsync(m->st.c + m->K * R, 0, (Ka - m->K) * R * 8, m->stream));
            CK(cudaMemsetAsync(m->st.D + m->K * R * R, 0, (Ka - m->K) * R * R * 8, m->stream));
        }
        CK(cudaMemcpyAsync(m->st.F, m->sw_F, (size_t)m->cfg.J * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        CK(cudaMemcpyAsync(m->st.G, m->sw_G, R * R * 8, cudaMemcpyDeviceToDevice, m->stream));
        s = run_update(m, b, X, m->cfg.lambda, false);
        if (s) return s;
    }
    return DASH_OK;
}

static dash_status update_common(dash_model *m, int64_t n_seg, const int64_t *ids,
                                 const int64_t *rp, const void *X, int64_t n_new) {
    if (!m->v_set) return fail(m, DASH_ESTATE, "V is not set (dash_set_factors)");
    if (m->broken) return fail(m, DASH_ESTATE, "model is unusable after a CUDA error");
    if (m->prof.pending.size() > 8192) prof_collect(m);
    BatchDev b;
    dash_status s = plan_batch(m, n_seg, ids, rp, m->K, n_new, X, true, &b);
    if (s) return s;
    CK(cudaMemsetAsync(m->d_err + 3, 0, sizeof(int), m->stream));
    m->K_prev = m->K;
    CK(cudaEventRecord(m->ev0, m->stream));
    const auto tl0 = std::chrono::steady_clock::now();
    const bool graph = m->use_graph && !m->prof.on;
    if (graph) CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    s = launch_sweeps(m, b, X);
    if (graph) {
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(m->stream, &g);
        if (s || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (s) return s;
            CK(ec);
        }
        if (m->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(m->gexec, g, &info) == cudaSuccess) {
                ++m->graph_updates;
            } else {                   // another launch topology: instantiate anew
                cudaGetLastError();
                cudaGraphExecDestroy(m->gexec);
                m->gexec = nullptr;
            }
        }
        if (!m->gexec) {
            const cudaError_t ei = cudaGraphInstantiate(&m->gexec, g, 0);
            cudaGraphDestroy(g);
            g = nullptr;
            CK(ei);
            ++m->graph_instantiations;
        }
        if (g) cudaGraphDestroy(g);
        CK(cudaGraphLaunch(m->gexec, m->stream));
    } else if (s) {
        return s;
    }
    if (m->prof.on) {
        m->prof.ms[KK_HOST_LAUNCH] +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tl0).count();
        m->prof.launches[KK_HOST_LAUNCH] += 1;
    }
    CK(cudaEventRecord(m->ev1, m->stream));
    m->K += n_new;
    m->last_N = b.N;
    m->has_last = true;
    m->xx_pending = true;
    m->xx_lam = m->cfg.lambda;
    m->last_X = X;
    m->last_ids.assign(ids, ids + n_seg);
    m->last_rp.assign(rp, rp + n_seg + 1);
    return DASH_OK;
}

static void clear_staging(dash_model *m) {
    m->st_slice.clear();
    m->st_row.assign(1, 0);
    m->st_rows = 0;
    m->st_new = 0;
}

// The model's stream waits for split host copies into the staging buffer.
static dash_status join_copies(dash_model *m) {
    if (m->copies_pending) {
        for (int i = 0; i < kCopyStreams; ++i) CK(cudaStreamWaitEvent(m->stream, m->copy_ev[i], 0));
        m->copies_pending = false;
    }
    return DASH_OK;
}

// After an update that read the staging buffer: mark it free once that work
// is done, and stage the next rows into the other buffer.
static dash_status flip_staging(dash_model *m) {
    CK(cudaEventRecord(m->buf_free[m->st_buf], m->stream));
    m->st_buf ^= 1;
    m->Xs = m->Xs_buf[m->st_buf];
    clear_staging(m);
    return DASH_OK;
}

extern "C" dash_status dash_update(dash_model *m) {
    if (!m) return DASH_EINVAL;
    const int64_t n_seg = m->st_segs();
    if (dash_status e = join_copies(m)) return e;
    dash_status s = update_common(m, n_seg, m->st_slice.data(), m->st_row.data(), m->Xs, m->st_new);
    if (s == DASH_OK) return flip_staging(m);
    return s;
}

extern "C" dash_status dash_update_device(dash_model *m, int64_t n_seg, const int64_t *slice_ids,
                                          const int64_t *row_ptr, const void *X) {
    if (!m) return DASH_EINVAL;
    if (m->st_segs() > 0) return fail(m, DASH_ESTATE, "rows are staged; call dash_update first");
    int64_t n_new = 0;
    dash_status s = check_csr(m, n_seg, slice_ids, row_ptr, m->K, &n_new);
    if (s) return s;
    const int64_t N = n_seg ? row_ptr[n_seg] : 0;
    if (N > m->cfg.max_rows) return fail(m, DASH_ENOMEM, "batch rows exceed max_rows");
    if (n_seg > m->cfg.max_segments) return fail(m, DASH_ENOMEM, "batch segments exceed max_segments");
    if (m->K + n_new > m->cfg.max_slices) return fail(m, DASH_ENOMEM, "slices would exceed max_slices");
    if (N > 0 && !X) return fail(m, DASH_EINVAL, "X is null");
    return update_common(m, n_seg, slice_ids, row_ptr, X, n_new);
}

static dash_status fit_common(dash_model *m, int64_t n_seg, const int64_t *ids,
                              const int64_t *rp, const void *X, int64_t n_new, int32_t n_iter) {
    if (n_iter < 1) return fail(m, DASH_EINVAL, "n_iter must be >= 1");
    if (m->K != 0) return fail(m, DASH_ESTATE, "fit_initial needs an empty model");
    if (!m->v_set) return fail(m, DASH_ESTATE, "V is not set (dash_set_factors)");
    if (m->broken) return fail(m, DASH_ESTATE, "model is unusable after a CUDA error");
    for (int64_t s = 0; s < n_seg; ++s)
        if (ids[s] < 0 || ids[s] >= n_new)
            return fail(m, DASH_EINVAL, "fit_initial takes new slices only");
    BatchDev b;
    dash_status s = plan_batch(m, n_seg, ids, rp, 0, n_new, X, true, &b);
    if (s) return s;
    CK(cudaMemsetAsync(m->d_err + 3, 0, sizeof(int), m->stream));
    m->K_prev = 0;
    CK(cudaEventRecord(m->ev0, m->stream));
    // iteration 1: the slices are new (S_k = I); later iterations: the same
    // rows with the helpers of the previous iteration dropped (λ = 0), which
    // is one static ALS iteration each (single batch ≡ static ALS).
    for (int it = 0; it < n_iter; ++it) {
        BatchDev bi = b;
        if (it > 0) bi.K_old = bi.K_all;     // no new slices any more
        s = run_update(m, bi, X, 0.0, it == 0);
        if (s) return s;
    }
    if (m->cfg.mode == DASH_MODE_Q) {
        // helpers of the final factors (L_k, Z_k of A_k = X_k V S_k Hᵀ), no sweep
        BatchDev bi = b;
        bi.K_old = bi.K_all;
        s = run_update_q(m, bi, X, 0.0, false, false);
        if (s) return s;
    } else {
        // c_k = vec(X_k)ᵀ(V ⊙ U_k) with the final V (Eq. 6), over every row
        BatchDev ball;
        s = plan_batch(m, n_seg, ids, rp, 0, n_new, X, false, &ball);
        if (s) return s;
        s = recompute_c(m, ball, X);
        if (s) return s;
    }
    CK(cudaEventRecord(m->ev1, m->stream));
    m->K = n_new;
    m->xx = 0.0;
    m->xx_valid = true;
    m->xx_pending = true;          // the last iteration's ||X||² is ||X_0||²
    m->xx_lam = 0.0;
    m->last_N = b.N;
    m->has_last = true;
    m->last_X = X;
    m->last_ids.assign(ids, ids + n_seg);
    m->last_rp.assign(rp, rp + n_seg + 1);
    return DASH_OK;
}

extern "C" dash_status dash_fit_initial(dash_model *m, int32_t n_iter) {
    if (!m) return DASH_EINVAL;
    if (dash_status e = join_copies(m)) return e;
    dash_status s = fit_common(m, m->st_segs(), m->st_slice.data(), m->st_row.data(), m->Xs,
                               m->st_new, n_iter);
    if (s == DASH_OK) return flip_staging(m);
    return s;
}

extern "C" dash_status dash_fit_initial_device(dash_model *m, int64_t n_seg,
                                               const int64_t *slice_ids, const int64_t *row_ptr,
                                               const void *X, int32_t n_iter) {
    if (!m) return DASH_EINVAL;
    if (m->st_segs() > 0) return fail(m, DASH_ESTATE, "rows are staged");
    int64_t n_new = 0;
    dash_status s = check_csr(m, n_seg, slice_ids, row_ptr, 0, &n_new);
    if (s) return s;
    const int64_t N = n_seg ? row_ptr[n_seg] : 0;
    if (N > m->cfg.max_rows) return fail(m, DASH_ENOMEM, "batch rows exceed max_rows");
    if (n_seg > m->cfg.max_segments) return fail(m, DASH_ENOMEM, "batch segments exceed max_segments");
    if (n_new > m->cfg.max_slices) return fail(m, DASH_ENOMEM, "slices would exceed max_slices");
    if (N > 0 && !X) return fail(m, DASH_EINVAL, "X is null");
    return fit_common(m, n_seg, slice_ids, row_ptr, X, n_new, n_iter);
}

// ---------------------------------------------------------------------------
// save / load: the resumable state of §3.2.1 (the helpers an update reads as
// "old"), with the configuration that sized the model
// ---------------------------------------------------------------------------
namespace {
constexpr char kSaveMagic[8] = {'D', 'A', 'S', 'H', 'S', 'A', 'V', '1'};

struct SaveHeader {
    char magic[8];
    int32_t version, mode, J, R, precision, input_dtype, n_sweeps, xx_valid;
    double lambda, pinv_rtol, xx;
    int64_t max_slices, max_rows, max_segments, max_staged_rows, K;
};

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

struct Arrays {
    std::vector<double> a[7];
};

// Sizes of the saved arrays: mode P {V, W, c, D, F, G}; mode Q {V, H, W, L,
// Y, E, B^{1/2}} (the eigenbasis and square root of B_k kept with L_k so that
// a resumed model continues bit for bit).
void array_sizes(int mode, int64_t J, int64_t R, int64_t K, size_t *n, int *count) {
    if (mode == DASH_MODE_P) {
        const size_t s[6] = {(size_t)(J * R), (size_t)(K * R), (size_t)(K * R), (size_t)(K * R * R),
                             (size_t)(J * R), (size_t)(R * R)};
        for (int i = 0; i < 6; ++i) n[i] = s[i];
        *count = 6;
    } else {
        const size_t s[7] = {(size_t)(J * R), (size_t)(R * R), (size_t)(K * R), (size_t)(K * R * R),
                             (size_t)(K * R * J), (size_t)(K * R * R), (size_t)(K * R * R)};
        for (int i = 0; i < 7; ++i) n[i] = s[i];
        *count = 7;
    }
}
}  // namespace

extern "C" dash_status dash_save(const dash_model *mc, const char *path) {
    dash_model *m = const_cast<dash_model *>(mc);
    if (!m) return DASH_EINVAL;
    if (!path) return fail(m, DASH_EINVAL, "path is null");
    if (!m->v_set) return fail(m, DASH_ESTATE, "V is not set: nothing to save");
    if (m->st_segs() > 0) return fail(m, DASH_ESTATE, "rows are staged; update first");
    CK(cudaStreamSynchronize(m->stream));
    if (dash_status sn = check_numeric(m)) return sn;
    fold_xx(m);
    const dash_config &c = m->cfg;
    SaveHeader h{};
    memcpy(h.magic, kSaveMagic, 8);
    h.version = 1;
    h.mode = c.mode;
    h.J = c.J;
    h.R = c.R;
    h.precision = c.precision;
    h.input_dtype = c.input_dtype;
    h.n_sweeps = c.n_sweeps;
    h.xx_valid = m->xx_valid ? 1 : 0;
    h.lambda = c.lambda;
    h.pinv_rtol = c.pinv_rtol;
    h.xx = m->xx;
    h.max_slices = c.max_slices;
    h.max_rows = c.max_rows;
    h.max_segments = c.max_segments;
    h.max_staged_rows = c.max_staged_rows;
    h.K = m->K;
    size_t n[7];
    int cnt = 0;
    array_sizes(c.mode, c.J, c.R, m->K, n, &cnt);
    Arrays A;
    for (int i = 0; i < cnt; ++i) A.a[i].resize(n[i]);
    dash_status s;
    if (c.mode == DASH_MODE_P) {
        s = dash_get_state_p(m, A.a[0].data(), A.a[1].data(), A.a[2].data(), A.a[3].data(), A.a[4].data(),
                             A.a[5].data());
    } else {
        s = dash_get_state_q(m, A.a[0].data(), A.a[1].data(), A.a[2].data(), A.a[3].data(), A.a[4].data());
        if (!s && m->K > 0) s = get_summ(m, A.a[5].data(), m->qE, n[5]);
        if (!s && m->K > 0) s = get_summ(m, A.a[6].data(), m->qBh, n[6]);
    }
    if (s) return s;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(m, DASH_EINVAL, "cannot open %s for writing", path);
    uint64_t hash = fnv1a(1469598103934665603ull, &h, sizeof h);
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;
    for (int i = 0; i < cnt && ok; ++i) {
        if (n[i] == 0) continue;
        ok = fwrite(A.a[i].data(), 8, n[i], f) == n[i];
        hash = fnv1a(hash, A.a[i].data(), n[i] * 8);
    }
    ok = ok && fwrite(&hash, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(m, DASH_EINVAL, "writing %s failed", path);
    return DASH_OK;
}

extern "C" dash_status dash_load(const char *path, void *stream, dash_model **out) {
    if (!path || !out) return DASH_EINVAL;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return DASH_EINVAL;
    SaveHeader h{};
    bool ok = fread(&h, sizeof h, 1, f) == 1 && memcmp(h.magic, kSaveMagic, 8) == 0 && h.version == 1 &&
              (h.mode == DASH_MODE_P || h.mode == DASH_MODE_Q) && h.J > 0 && h.R > 0 && h.R <= kMaxR &&
              h.K >= 0 && h.K <= h.max_slices;
    size_t n[7] = {};
    int cnt = 0;
    Arrays A;
    uint64_t hash = fnv1a(1469598103934665603ull, &h, sizeof h);
    if (ok) {
        array_sizes(h.mode, h.J, h.R, h.K, n, &cnt);
        for (int i = 0; i < cnt && ok; ++i) {
            A.a[i].resize(n[i]);
            if (n[i] == 0) continue;
            ok = fread(A.a[i].data(), 8, n[i], f) == n[i];
            hash = fnv1a(hash, A.a[i].data(), n[i] * 8);
        }
        uint64_t stored = 0;
        ok = ok && fread(&stored, 8, 1, f) == 1 && stored == hash;
    }
    fclose(f);
    if (!ok) return DASH_EINVAL;
    dash_config c;
    dash_config_default(&c, h.J, h.R, h.lambda);
    c.mode = h.mode;
    c.precision = h.precision;
    c.input_dtype = h.input_dtype;
    c.n_sweeps = h.n_sweeps;
    c.pinv_rtol = h.pinv_rtol;
    c.max_slices = h.max_slices;
    c.max_rows = h.max_rows;
    c.max_segments = h.max_segments;
    c.max_staged_rows = h.max_staged_rows;
    c.stream = stream;
    dash_model *m = nullptr;
    dash_status s = dash_init(&c, &m);
    if (s) return s;
    if (h.mode == DASH_MODE_P) {
        s = dash_set_state_p(m, h.K, A.a[0].data(), A.a[1].data(), A.a[2].data(), A.a[3].data(),
                             A.a[4].data(), A.a[5].data());
    } else {
        s = dash_set_state_q(m, h.K, A.a[0].data(), A.a[1].data(), A.a[2].data(), A.a[3].data(),
                             A.a[4].data());
        if (!s && h.K > 0) s = put_summ(m, m->qE, A.a[5].data(), n[5]);
        if (!s && h.K > 0) s = put_summ(m, m->qBh, A.a[6].data(), n[6]);
    }
    if (s) {
        dash_destroy(m);
        return s;
    }
    m->xx = h.xx;
    m->xx_valid = h.xx_valid != 0;
    *out = m;
    return DASH_OK;
}
