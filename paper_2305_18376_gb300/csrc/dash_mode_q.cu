// Launch sequence of one constrained-mode (Q) update on the model's stream:
// the A rows, the λ-weighted summaries Z_k and L_k, T_k = (L_kᵀL_k)^{-1/2},
// one CP-ALS sweep H → V → W, the new Q rows and the batch residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "dash_host.cuh"
#include "dash_tmap.cuh"

namespace dash {

// Mode Q: one update (sweep = true) or, for the end of a static fit, the
// summaries of the current factors alone (sweep = false: L_k, Y_k, the new
// Q rows and the residual; factors untouched).
static QDev make_qdev(dash_model *m, double lam) {
    QDev q;
    q.J = m->cfg.J;
    q.R = m->cfg.R;
    q.lam = lam;
    q.rtol = m->rtol;
    q.V = m->st.V;
    q.H = m->qH;
    q.W = m->st.W;
    q.L = m->qL;
    q.E = m->qE;
    q.Bh = m->qBh;
    q.C = m->qC;
    q.Gam = m->st.Gam;
    q.err = m->d_err;
    q.phase = m->prof.phases && m->prof.d_phase ? m->prof.d_phase + 7 : nullptr;
    return q;
}

// Warps per CTA of k_q_lt: as many per-warp workspaces as fit in 212 KB.
template <class S>
static int q_lt_warps(int R) {
    const size_t wb = q_lt_warp_bytes<S>(R);
    return (int)std::min<size_t>(8, std::max<size_t>(1, (size_t)(212 * 1024) / wb));
}

template <class S, typename T>
static dash_status launch_lt(dash_model *m, const BatchDev &b, const QDev &q, const T *A, T *Qrows,
                             int mode) {
    const int R = m->cfg.R;
    const int nw = q_lt_warps<S>(R);
    const size_t smem = (size_t)nw * q_lt_warp_bytes<S>(R);
    const int grid = std::max(1, std::min((b.K_all + nw - 1) / nw, 4 * m->n_sm));
    // rotation threshold on |γ|/√(αβ): FP64 and FP32 a few units of their
    // roundoff; double-float 1e-10, four orders below what one FP32 rounding
    // of the mixed path's inputs moves the eigenvectors by on these slices
    // (its sweeps also stop early once a sweep starts below sqrt(1e-10)/2)
    const float jtol = std::is_same<S, double>::value ? 1e-15f
                     : std::is_same<S, float>::value ? 3e-7f : 1e-10f;
    CK(cudaFuncSetAttribute(k_q_lt<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    m->prof.q_lt_warps = (double)grid * nw;
    LAUNCH(KK_Q_LT, (k_q_lt<S, T><<<grid, 32 * nw, smem, m->stream>>>(b, q, A, Qrows, mode, 6, jtol)));
    return DASH_OK;
}

template <typename TI, typename T, class S>
static dash_status launch_update_q(dash_model *m, const BatchDev &b, const void *Xv, double lam,
                                   bool begin_new, bool sweep) {
    const int J = m->cfg.J, R = m->cfg.R;
    cudaStream_t st = m->stream;
    const TI *X = (const TI *)Xv;
    const int64_t N = b.N;
    const int n_new = b.K_all - b.K_old;
    const QDev q = make_qdev(m, lam);
    T *Y = (T *)m->qY;
    T *A = (T *)m->qA;
    T *Qrows = (T *)m->U;
    if (begin_new && n_new > 0) {
        const int64_t tot = (int64_t)n_new * R * (1 + 3 * R + J);
        LAUNCH(KK_Q_BEGIN, (k_q_begin_new<S, T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
                               m->st.W, m->qL, m->qE, m->qBh, Y, b.K_old, n_new, R, J)));
    }
    if (N > 0) {
        LAUNCH(KK_ROWMAP, k_rowmap<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(b));
        // P = X V: on tcgen05 MMAs (the mode-P X·Q_V pass with V's TF32 slabs
        // in place of Q_V's) when the batch's rows form one run from row 0,
        // else the SIMT kernel
        bool tc05 = false;
        if constexpr (std::is_same<T, float>::value && std::is_same<TI, float>::value) {
            CUtensorMap tmx;
            if (m->xu_nst > 0 && b.n_runs == 1 && m->h_run_row0[0] == 0 && b.N_gen == N)
                tc05 = x_tensor_map(&tmx, (const float *)X, J, N, 32, 128, true);
            if (tc05) {
                const int nslab = xu_slabs(J);
                LAUNCH(KK_QV_TF32, k_qv_tf32<<<(nslab * 2048 + 255) / 256, 256, 0, st>>>(
                                       (const float *)m->VT, J, R, m->qv_slabs));
                const int n_xn = (int)std::min<int64_t>(m->n_sm, (N + 127) / 128);
                XuArgs xa{m->qv_slabs, (float *)m->P, m->xn_part, m->d_err, N, 0, J, R,
                          m->xr_nst > 0 ? m->xr_nst : m->xu_nst, m->wait_limit, 0, nullptr};
                if (m->xr_nst > 0) {
                    const size_t smem = xr_smem(J, m->xr_nst);
                    CK(cudaFuncSetAttribute(k_xq_umma_rq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                    LAUNCH(KK_XQ_UMMA, k_xq_umma_rq<<<n_xn, XR_THREADS, smem, st>>>(tmx, xa));
                } else {
                    const size_t smem = xu_smem(J, m->xu_nst);
                    CK(cudaFuncSetAttribute(k_xq_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                    LAUNCH(KK_XQ_UMMA, k_xq_umma<<<n_xn, XU_THREADS, smem, st>>>(tmx, xa));
                }
            }
        }
        if (!tc05) {
            const int n_xn = (int)((N + XV_ROWS - 1) / XV_ROWS);
            LAUNCH(KK_XV, (k_xv<TI, T><<<n_xn, 256, 0, st>>>(X, b, J, R, (const T *)m->VT, (T *)m->P,
                                                             m->xn_part)));
        }
        if (R <= 32) {
            const unsigned ga = (unsigned)std::min<int64_t>((N + 7) / 8, (int64_t)m->n_sm * 16);
            LAUNCH(KK_Q_AROWS, (k_q_arows_w<T><<<ga, 256, 0, st>>>(N, R, b.row_slice, (const T *)m->P,
                                                                    m->st.W, m->qH, A)));
        } else {
            LAUNCH(KK_Q_AROWS, (k_q_arows<T><<<(unsigned)((N * R + 255) / 256), 256, 0, st>>>(
                                   N, R, b.row_slice, (const T *)m->P, m->st.W, m->qH, A)));
        }
    }
    dash_status s = launch_lt<S, T>(m, b, q, A, Qrows, 0);
    if (s) return s;
    const int gy = std::max(1, std::min(b.K_all, m->q_lt_max));
    if (b.K_all > 0) {
        const size_t ysm = q_y_smem<T>(R);
        if (R <= 32) {
            CK(cudaFuncSetAttribute(k_q_y<TI, T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm));
            LAUNCH(KK_Q_Y, (k_q_y<TI, T, 32><<<gy, QZ_THREADS, ysm, st>>>(b, q, X, Qrows, Y, (const T *)m->VT,
                                                                           m->qMH, m->qWWp)));
        } else {
            CK(cudaFuncSetAttribute(k_q_y<TI, T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm));
            LAUNCH(KK_Q_Y, (k_q_y<TI, T, 64><<<gy, QZ_THREADS, ysm, st>>>(b, q, X, Qrows, Y, (const T *)m->VT,
                                                                           m->qMH, m->qWWp)));
        }
    } else {
        CK(cudaMemsetAsync(m->qMH, 0, (size_t)R * R * 8, st));
        CK(cudaMemsetAsync(m->qWWp, 0, (size_t)R * R * 8, st));
    }
    const int ld = R + 1;
    if (sweep) {
        // the per-CTA partials summed across SMs first (one warp summing them
        // serially was latency-bound), then H and the pseudo-inverses
        const int nyb = b.K_all > 0 ? gy : 1;
        if (nyb > 1) {
            const int g = (int)std::min<int64_t>(((int64_t)R * R + 255) / 256, m->n_sm);
            LAUNCH(KK_Q_PSUM, (k_q_psum<<<g, 256, 0, st>>>(m->qMH, nyb, (int64_t)R * R)));
            LAUNCH(KK_Q_PSUM, (k_q_psum<<<g, 256, 0, st>>>(m->qWWp, nyb, (int64_t)R * R)));
        }
        LAUNCH(KK_Q_H, (k_q_h<<<1, 32, (size_t)(4 * R * ld + R) * 8, st>>>(m->qMH, m->qWWp, 1, q,
                                                                             m->qWW, m->qPV)));
        const int gv = std::max(1, std::min(b.K_all, m->q_vslots));
        if (R <= 32)
            LAUNCH(KK_Q_VPART, (k_q_vpart<T, 32><<<gv, QV_THREADS, 0, st>>>(b.K_all, q, Y, m->qslots)));
        else
            LAUNCH(KK_Q_VPART, (k_q_vpart<T, 64><<<gv, QV_THREADS, 0, st>>>(b.K_all, q, Y, m->qslots)));
        if (gv > 1) {
            const int g = (int)std::min<int64_t>(((int64_t)J * R + 255) / 256, 2 * m->n_sm);
            LAUNCH(KK_Q_PSUM, (k_q_psum<<<g, 256, 0, st>>>(m->qslots, gv, (int64_t)J * R)));
        }
        LAUNCH(KK_Q_V, (k_q_v<T><<<(J + 7) / 8, 256, 0, st>>>(m->qslots, 1, m->qPV, J, R, m->st.V,
                                                               (T *)m->VT)));
        LAUNCH(KK_GAMMA, k_gamma<<<(R * R + 7) / 8, 256, 0, st>>>(m->st.V, J, R, m->st.Gam, nullptr));
        LAUNCH(KK_Q_PW, (k_q_pw<<<1, 32, (size_t)(3 * R * ld + R) * 8, st>>>(q, m->qPW)));
        if (b.K_all > 0) {
            const int gw = std::min(b.K_all, 4 * m->n_sm);
            const size_t wsm = q_w_smem<T>(R);
            CK(cudaFuncSetAttribute(k_q_w<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm));
            LAUNCH(KK_Q_W, (k_q_w<T><<<gw, QZ_THREADS, wsm, st>>>(b.K_all, q, Y, (const T *)m->VT, m->qPW)));
        }
    }
    int go = 1;
    if (N > 0) {
        go = (int)std::min<int64_t>((N + 7) / 8, m->q_out_max);
        const size_t osm = q_out_smem<T>(R, J);
        CK(cudaFuncSetAttribute(k_q_out<TI, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osm));
        LAUNCH(KK_Q_OUT, (k_q_out<TI, T><<<go, 256, osm, st>>>(N, q, b.row_slice, X, Qrows,
                                                              (const T *)m->VT, m->qfit)));
    } else {
        CK(cudaMemsetAsync(m->qfit, 0, 2 * 8, st));
    }
    LAUNCH(KK_Q_FIT, (k_q_fit<<<1, 32, 0, st>>>(m->qfit, go, m->st.gam_ok, m->fit)));
    CK(cudaMemcpyAsync(m->h_fit, m->fit, 4 * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(m->h_err, m->d_err, kErrSlots * sizeof(int), cudaMemcpyDeviceToHost, st));
    return DASH_OK;
}

dash_status run_update_q(dash_model *m, const BatchDev &b, const void *X, double lam,
                         bool begin_new, bool sweep) {
    const bool f64in = m->cfg.input_dtype == DASH_F64;
    if (m->tsize == 8) {
        return f64in ? launch_update_q<double, double, double>(m, b, X, lam, begin_new, sweep)
                     : launch_update_q<float, double, double>(m, b, X, lam, begin_new, sweep);
    }
    return f64in ? launch_update_q<double, float, df>(m, b, X, lam, begin_new, sweep)
                 : launch_update_q<float, float, df>(m, b, X, lam, begin_new, sweep);
}

dash_status prepare_q(dash_model *m) {
    if (m->K == 0) return DASH_OK;
    BatchDev b{};
    b.K_all = (int)m->K;
    b.K_old = (int)m->K;
    const QDev q = make_qdev(m, m->cfg.lambda);
    if (m->tsize == 8) return launch_lt<double, double>(m, b, q, nullptr, nullptr, 1);
    return launch_lt<df, float>(m, b, q, nullptr, nullptr, 1);
}

}  // namespace dash
