// Launch sequence of one mode-P update (Algorithm 1) on the model's stream:
// the fused row kernel over tiles of single-segment slices, the chunked path
// for large or split slices, the general kernels, and the global reductions
// and solves (Eqs. 11-21).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "dash_host.cuh"
#include "dash_tmap.cuh"

namespace dash {

// Time the X·Q_V pass variants on this batch and keep the fastest: the
// resident-Q_V kernel at every ring depth from 2 to the deepest that fits,
// then the streamed-slab kernel.  Every variant writes the same P' and ‖X‖²
// partials (the same MMAs in the same order), so the last one launched
// leaves correct outputs either way.  Synchronises the stream once.
static dash_status autotune_xq(dash_model *m, const CUtensorMap &tmx, XuArgs xa, int n_xn, cudaStream_t st) {
    const int J = m->cfg.J;
    struct Cand { bool rq; int nst; };
    Cand c[8];
    int nc = 0;
    for (int d = 2; d <= xr_stages(J) && nc < 7; ++d) c[nc++] = {true, d};
    if (m->xu_nst > 0) c[nc++] = {false, m->xu_nst};
    m->xu_tuned = true;
    m->xu_tune_n = nc;
    if (nc < 2) {
        m->xu_tune_best = nc - 1;
        return DASH_OK;
    }
    cudaEvent_t ev[16];
    for (int i = 0; i < 2 * nc; ++i) CK(cudaEventCreate(&ev[i]));
    // every candidate runs once untimed (its first launch carries one-time
    // costs), then once timed
    for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < nc; ++i) {
        xa.nst = c[i].nst;
        if (pass == 1) CK(cudaEventRecord(ev[2 * i], st));
        if (c[i].rq) {
            const size_t smem = xr_smem(J, c[i].nst);
            CK(cudaFuncSetAttribute(k_xq_umma_rq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            LAUNCH(KK_XQ_UMMA, k_xq_umma_rq<<<n_xn, XR_THREADS, smem, st>>>(tmx, xa));
        } else {
            const size_t smem = xu_smem(J, c[i].nst);
            CK(cudaFuncSetAttribute(k_xq_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            LAUNCH(KK_XQ_UMMA, k_xq_umma<<<n_xn, XU_THREADS, smem, st>>>(tmx, xa));
        }
        if (pass == 1) CK(cudaEventRecord(ev[2 * i + 1], st));
    }
    CK(cudaEventSynchronize(ev[2 * nc - 1]));
    int best = 0;
    for (int i = 0; i < nc; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        m->xu_tune_ms[i] = ms;
        if (ms < m->xu_tune_ms[best]) best = i;
    }
    for (int i = 0; i < 2 * nc; ++i) cudaEventDestroy(ev[i]);
    m->xu_tune_best = best;
    m->xr_nst = c[best].rq ? c[best].nst : 0;
    return DASH_OK;
}

template <typename TI, typename T>
static dash_status launch_update_p(dash_model *m, const BatchDev &b, const void *Xv, double lam,
                                   bool begin_new) {
    const int J = m->cfg.J, R = m->cfg.R;
    cudaStream_t st = m->stream;
    const TI *X = (const TI *)Xv;
    StateDev s = m->st;
    s.lam = lam;
    const int64_t N = b.N;
    const int64_t Ng = b.N_gen;
    const int n_new = b.K_all - b.K_old;
    constexpr bool DF = std::is_same<T, float>::value;
    if (begin_new && n_new > 0) {
        const int64_t tot = (int64_t)n_new * R * (R + 2);
        LAUNCH(KK_BEGIN_NEW, k_begin_new<<<(tot + 255) / 256, 256, 0, st>>>(s.W, s.c, s.D, b.K_old, n_new, R));
    }
    // fused row kernel over the tiles of single-segment slices
    int g_f = 0;
    if constexpr (std::is_same<T, float>::value && std::is_same<TI, float>::value) {
        if (m->fused_active) {
            // the Cholesky QR of V: computed at the end of the previous update
            // unless the state was set since
            if (!m->vqr_fresh) {
                const size_t qsm = (size_t)(2 * R * (R + 1) + R + 1) * 8;
                LAUNCH(KK_VTILDE, k_vqr<<<1, 32, qsm, st>>>(s.Gam, R, m->rtol, m->RV, m->Linv, m->GPf,
                                                            m->Gdf, s.gam_ok));
                m->vqr_fresh = true;
            }
            LAUNCH(KK_QV, k_qv<<<(J + 7) / 8, 256, 0, st>>>(s.V, m->Linv, J, R, m->QV));
        }
        if (m->fused_active && m->n_tiles > 0) {
            g_f = std::min(m->n_sm, m->n_tiles);
            FusedArgs fa{};
            fa.X = X;
            fa.J = J;
            fa.R = R;
            fa.lam = lam;
            fa.lam_hi = (float)lam;
            fa.lam_lo = (float)(lam - (double)fa.lam_hi);
            fa.lam_on = lam != 0.0;
            fa.rtol = m->rtol;
            fa.V32 = m->QV;
            fa.GPf = m->GPf;
            fa.RV = m->RV;
            fa.Gdf = m->Gdf;
            fa.Gam = s.Gam;
            fa.gam_ok = s.gam_ok;
            fa.n_tiles = m->n_tiles;
            fa.tile_s0 = m->d_tile_s0;
            fa.tile_s1 = m->d_tile_s1;
            fa.seg_row = b.seg_row;
            fa.seg_slice = b.seg_slice;
            fa.W = s.W;
            fa.c = reinterpret_cast<df *>(s.c);
            fa.D = reinterpret_cast<df *>(s.D);
            fa.U = (float *)m->U;
            fa.Fslot = (float *)m->Fpart;
            fa.Gpart = m->Gpart;
            fa.xn_part = m->xn_part;
            fa.wsp = m->wsp;
            fa.err = m->d_err;
            fa.phase_cycles = m->prof.phases && m->prof.d_phase ? m->prof.d_phase : nullptr;
            const size_t smem = fu_smem_bytes(J);
            if (m->cfg.precision == DASH_PREC_F16X3) {
                CK(cudaFuncSetAttribute(k_rows_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                LAUNCH(KK_ROWS_FUSED, k_rows_fused<true><<<g_f, FU_THREADS, smem, st>>>(fa));
            } else {
                CK(cudaFuncSetAttribute(k_rows_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                LAUNCH(KK_ROWS_FUSED, k_rows_fused<false><<<g_f, FU_THREADS, smem, st>>>(fa));
            }
        }
    }
    int n_xn = 0;
    // the tcgen05 passes of the split pipeline: their tensor maps over X
    CUtensorMap tmx, tmxf;
    bool tc05 = false;
    // P = X V for the general kernels; P' = X Q_V for the chunked path
    const T *Vmul = (const T *)m->VT;
    if constexpr (std::is_same<T, float>::value) {
        if (m->fused_active) Vmul = (const T *)m->QV;
    }
    bool split = false;
    if constexpr (std::is_same<T, float>::value && std::is_same<TI, float>::value) split = m->split_active;
    if (Ng > 0) {
        LAUNCH(KK_ROWMAP, k_rowmap<<<(N + 255) / 256, 256, 0, st>>>(b));
        if (split && m->xu_nst > 0 && m->row_path != DASH_ROWS_SPLIT_WARP && b.n_runs == 1) {
            const float *X0 = (const float *)X + m->h_run_row0[0] * J;
            tc05 = x_tensor_map(&tmx, X0, J, Ng, 32, 128, true) &&
                   x_tensor_map(&tmxf, X0, J, Ng, 128, FB_ROWS, false);
        }
        if (tc05) {
            // P' = X Q_V on tcgen05 MMAs, X tiles by TMA, Q_V as TF32 slabs
            const int nslab = xu_slabs(J);
            LAUNCH(KK_QV_TF32, k_qv_tf32<<<(nslab * 2048 + 255) / 256, 256, 0, st>>>(m->QV, J, R, m->qv_slabs));
            n_xn = (int)std::min<int64_t>(m->n_sm, (Ng + 127) / 128);
            XuArgs xa{m->qv_slabs, (float *)m->P, m->xn_part + g_f, m->d_err, Ng, m->h_run_row0[0],
                      J, R, m->xr_nst > 0 ? m->xr_nst : m->xu_nst, m->wait_limit, m->inject_wait_fault,
                      m->prof.phases && m->prof.d_phase ? m->prof.d_phase + 15 : nullptr};
            m->inject_wait_fault = 0;
            if (m->autotune && !m->xu_tuned && !m->use_graph && xa.skip_first_copy == 0) {
                if (dash_status e = autotune_xq(m, tmx, xa, n_xn, st)) return e;
                xa.nst = m->xr_nst > 0 ? m->xr_nst : m->xu_nst;
            }
            if (m->xr_nst > 0) {
                // Q_V resident in shared memory, X released after conversion
                const size_t smem = xr_smem(J, m->xr_nst);
                CK(cudaFuncSetAttribute(k_xq_umma_rq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                LAUNCH(KK_XQ_UMMA, k_xq_umma_rq<<<n_xn, XR_THREADS, smem, st>>>(tmx, xa));
                m->prof.xq_warps = (double)n_xn * (XR_THREADS / 32);
                m->prof.xu_conv_warps = 4.0;
            } else {
                const size_t smem = xu_smem(J, m->xu_nst);
                CK(cudaFuncSetAttribute(k_xq_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                LAUNCH(KK_XQ_UMMA, k_xq_umma<<<n_xn, XU_THREADS, smem, st>>>(tmx, xa));
                m->prof.xq_warps = (double)n_xn * (XU_THREADS / 32);
                m->prof.xu_conv_warps = 4.0 * XU_CONV_GROUPS;
            }
            m->prof.xu_ctas = n_xn;
        } else if (split) {
            // P' = X Q_V on the tensor cores, Q_V pre-split into fragments
            const int nfr = ((J + 15) / 16) * ((R + 7) / 8) * 32;
            LAUNCH(KK_XQ_PREP, k_xq_bscale<<<1, 32, 0, st>>>(m->QV, J * R, m->xq_bexp));
            LAUNCH(KK_XQ_PREP, k_xq_bfrag<<<(nfr + 255) / 256, 256, 0, st>>>(m->QV, J, R, m->xq_bexp,
                                                                            m->xq_frag));
            const int64_t ntile = (Ng + 15) / 16;
            n_xn = (int)std::min<int64_t>(m->n_sm, (ntile + XQ_WARPS - 1) / XQ_WARPS);
            const size_t smem = xq_smem(J, R);
            CK(cudaFuncSetAttribute(k_xq_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            LAUNCH(KK_XQ_TC, k_xq_tc<<<n_xn, XQ_THREADS, smem, st>>>((const float *)X, b, J, R, m->xq_frag,
                                                                     m->xq_bexp, (float *)m->P,
                                                                     m->xn_part + g_f, m->xe, m->d_err,
                                                                     m->prof.phases && m->prof.d_phase ? m->prof.d_phase + 11 : nullptr));
            m->prof.xq_warps = (double)n_xn * XQ_WARPS;
        } else {
            n_xn = (int)((Ng + XV_ROWS - 1) / XV_ROWS);
            LAUNCH(KK_XV, k_xv<TI, T><<<n_xn, 256, 0, st>>>(X, b, J, R, Vmul, (T *)m->P,
                                                            m->xn_part + g_f));
        }
    }
    int nsb = 0;
    bool finished = false;
    if constexpr (std::is_same<T, float>::value && std::is_same<TI, float>::value) {
        if (m->fused_active) {
            // chunks of big / split slices, then every remaining slice's finish
            FusedArgs fa{};
            fa.J = J;
            fa.R = R;
            fa.lam = lam;
            fa.lam_hi = (float)lam;
            fa.lam_lo = (float)(lam - (double)fa.lam_hi);
            fa.lam_on = lam != 0.0;
            fa.rtol = m->rtol;
            fa.Gdf = m->Gdf;
            fa.GPf = m->GPf;
            fa.RV = m->RV;
            fa.Gam = s.Gam;
            fa.gam_ok = s.gam_ok;
            fa.W = s.W;
            fa.Wf = split ? m->Wf : nullptr;
            fa.c = reinterpret_cast<df *>(s.c);
            fa.D = reinterpret_cast<df *>(s.D);
            fa.U = (float *)m->U;
            fa.wsp = m->wsp;
            fa.err = m->d_err;
            BigArgs bg{};
            bg.Y = (const float *)m->P;
            bg.ch_row0 = m->d_ch_row0;
            bg.ch_n = m->d_ch_n;
            bg.ch_k = m->d_ch_k;
            bg.n_chunks = m->n_chunks;
            bg.fin_k = m->d_fin_k;
            bg.fin_c0 = m->d_fin_c0;
            bg.n_fin = m->n_fin;
            bg.dpart = m->dpart;
            // both grids stay within the 2-CTAs-per-SM workspace (persistent warps)
            if (m->n_chunks > 0) {
                const int gb = std::min(2 * m->n_sm, (m->n_chunks + FU_WARPS - 1) / FU_WARPS);
                if (split && (R % 2) == 0)
                    LAUNCH(KK_BIG_B, k_big_b_tc<<<gb, 256, 0, st>>>(fa, bg));
                else
                    LAUNCH(KK_BIG_B, k_big_b<<<gb, 256, 0, st>>>(fa, bg));
            }
            if (m->n_fin > 0) {
                nsb = std::min(kBigCBlocksPerSM * m->n_sm, (m->n_fin + FU_WARPS - 1) / FU_WARPS);
                // the whole unified L1/shared array as shared memory, so that
                // kBigCBlocksPerSM CTAs fit on an SM
                CK(cudaFuncSetAttribute(k_big_c, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
                fa.phase_cycles = m->prof.phases && m->prof.d_phase ? m->prof.d_phase + 20 : nullptr;
                LAUNCH(KK_BIG_C, k_big_c<<<nsb, 256, 0, st>>>(fa, bg, m->Gpart + (size_t)g_f * R * R));
                fa.phase_cycles = nullptr;
                m->prof.bc_warps = (double)nsb * 8;
            }
            finished = true;
        }
    }
    if (!finished) {
        // the general kernel reads Γ⁺
        if (!m->gamp_fresh) {
            if (dash_status e = launch_pinv(m, s.Gam, s.GamP, s.gam_ok, nullptr)) return e;
            m->gamp_fresh = true;
        }
        // per-slice work for slices the fused kernel did not finish
        const int nw = sl_warps(R);
        const size_t smem = (size_t)nw * sl_warp_doubles(R) * 8;
        nsb = (int)std::min<int64_t>((b.K_all + nw - 1) / nw, kSliceBlocksMax);
        if (nsb < 1) nsb = 1;
        CK(cudaFuncSetAttribute(k_slices<T, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LAUNCH(KK_SLICES, k_slices<T, DF><<<nsb, 32 * nw, smem, st>>>(b, s, (const T *)m->P, (T *)m->U,
                                                                      m->Gpart + (size_t)g_f * R * R));
    }
    // F partials of the general rows
    int nfb = 0;
    if (Ng > 0 && tc05) {
        // the F partials on tcgen05 MMAs, Ũ = U ∘ w_new built in the kernel:
        // about one CTA per SM, row chunks × 128-column tiles
        const int nmt = (J + 127) / 128;
        nfb = std::max(1, m->n_sm / nmt);
        const int64_t rpc = ((Ng + nfb - 1) / nfb + FB_ROWS - 1) / FB_ROWS * FB_ROWS;
        nfb = (int)((Ng + rpc - 1) / rpc);
        if (g_f + nfb > m->n_fb_max) return fail(m, DASH_ECUDA, "internal: F partials exceed their buffer");
        FbArgs fb{b, (const float *)m->U, m->Wf, (int64_t)(m->n_fb_max - g_f),
                  (float *)m->Fpart + (size_t)g_f * J * R, m->d_err, Ng, rpc, J, R, m->wait_limit};
        CK(cudaFuncSetAttribute(k_f_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem()));
        LAUNCH(KK_F_UMMA, k_f_umma<<<dim3(nfb, nmt), FB_THREADS, fb_smem(), st>>>(tmxf, fb));
        m->prof.ft_warps = (double)nfb * nmt * (FB_THREADS / 32);
    } else if (Ng > 0 && split) {
        // Ũ = U ∘ w_new, then the F partials on the tensor cores: one CTA per
        // SM, rows in equal shares
        const int NT = (R + 7) / 8;
        nfb = (int)std::min<int64_t>(m->n_sm, (Ng + 127) / 128);
        const int64_t rpc = ((Ng + nfb - 1) / nfb + 15) / 16 * 16;
        nfb = (int)((Ng + rpc - 1) / rpc);
        dim3 grid(nfb, (J + FT_JCTA - 1) / FT_JCTA);
        float *Fo = (float *)m->Fpart + (size_t)g_f * J * R;
        const float *Xf = (const float *)X;
        m->prof.ft_warps = (double)grid.x * grid.y * FT_WARPS;
        const unsigned nug = (unsigned)((Ng + 127) / 128);
        unsigned long long *pc = m->prof.phases && m->prof.d_phase ? m->prof.d_phase + 13 : nullptr;
        switch (NT) {
#define FTC(n)                                                                                       \
    case n:                                                                                          \
        LAUNCH(KK_UTILDE, k_utilde<n><<<nug, 256, 0, st>>>(b, R, (const float *)m->U, m->Wf, m->xe, \
                                                            m->Ut));                                 \
        CK(cudaFuncSetAttribute(k_f_tc<n>, cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                                (int)ft_smem(n)));                                                   \
        LAUNCH(KK_F_TC, k_f_tc<n><<<grid, FT_THREADS, ft_smem(n), st>>>(Xf, b, J, R, m->Ut, rpc,    \
                                                                        Fo, m->d_err, pc));          \
        break;
            FTC(1)
            FTC(2)
            FTC(3)
            FTC(4)
#undef FTC
        }
    } else if (Ng > 0) {
        const int nby = (J + F_JB - 1) / F_JB;
        nfb = (int)std::min<int64_t>(std::max<int64_t>(1, (2 * 152 * 4) / nby), (Ng + F_RC - 1) / F_RC);
        nfb = std::min(nfb, kFBlocksMax);
        int64_t rpc = (Ng + nfb - 1) / nfb;
        rpc = (rpc + F_RC - 1) / F_RC * F_RC;
        nfb = (int)((Ng + rpc - 1) / rpc);
        dim3 grid(nfb, nby);
        LAUNCH(KK_F, k_f<TI, T><<<grid, 256, 0, st>>>(X, b, J, R, (const T *)m->U, s.W, rpc,
                                                     (T *)m->Fpart + (size_t)g_f * J * R));
    }
    LAUNCH(KK_F_REDUCE, k_f_reduce<T><<<((int64_t)J * R + 255) / 256, 256, 0, st>>>((const T *)m->Fpart, g_f + nfb, J, R, lam,
                                                                s.F, m->Finc, m->d_err + 3));
    LAUNCH(KK_G_REDUCE, k_g_reduce<<<(R * R + 7) / 8, 256, 0, st>>>(m->Gpart, g_f + nsb, R, lam, s.G, m->Ginc,
                                                                  m->d_err + 3));
    if (dash_status e = launch_pinv(m, s.G, m->GP, nullptr, m->d_err + 3)) return e;
    LAUNCH(KK_VUPDATE, k_vupdate<T><<<(J + 7) / 8, 256, 0, st>>>(s.F, m->GP, m->Finc, J, R, s.V, (T *)m->VT,
                                               m->cross_part, m->d_err + 3, m->d_err + 2));
    LAUNCH(KK_GAMMA, k_gamma<<<(R * R + 7) / 8, 256, 0, st>>>(s.V, J, R, s.Gam, m->d_err + 3));
    if (m->fused_ok) {
        // mixed path: the Cholesky QR of the new V for the next update (it also
        // decides whether Γ is nonsingular); Γ⁺ only if an update needs it
        const size_t qsm = (size_t)(2 * R * (R + 1) + R + 1) * 8;
        LAUNCH(KK_VTILDE, k_vqr<<<1, 32, qsm, st>>>(s.Gam, R, m->rtol, m->RV, m->Linv, m->GPf, m->Gdf,
                                                    s.gam_ok));
        m->vqr_fresh = true;
        m->gamp_fresh = false;
    } else {
        if (dash_status e = launch_pinv(m, s.Gam, s.GamP, s.gam_ok, m->d_err + 3)) return e;
        m->gamp_fresh = true;
        m->vqr_fresh = false;
    }
    LAUNCH(KK_FITNESS, k_fitness<<<1, 32, 0, st>>>(m->xn_part, g_f + n_xn, m->cross_part, (J + 7) / 8, s.Gam, m->Ginc, R,
                                s.gam_ok, m->fit));
    CK(cudaMemcpyAsync(m->h_fit, m->fit, 4 * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(m->h_err, m->d_err, kErrSlots * sizeof(int), cudaMemcpyDeviceToHost, st));
    return DASH_OK;
}

template <typename TI, typename T>
static dash_status launch_recompute_c(dash_model *m, const BatchDev &b0, const void *Xv) {
    const int J = m->cfg.J, R = m->cfg.R;
    constexpr bool DF = std::is_same<T, float>::value;
    const BatchDev &b = b0;     // planned without fused tiles: every row is general
    if (b.N > 0) {
        const int n_xn = (int)((b.N + XV_ROWS - 1) / XV_ROWS);
        LAUNCH(KK_XV, k_xv<TI, T><<<n_xn, 256, 0, m->stream>>>((const TI *)Xv, b, J, R, (const T *)m->VT,
                                                  (T *)m->P, m->xn_part));
    }
    const int nb = (b.K_all + 7) / 8;
    LAUNCH(KK_C_RECOMPUTE, k_c_recompute<T, DF><<<nb > 0 ? nb : 1, 256, 0, m->stream>>>(b, (const T *)m->P, (const T *)m->U, R,
                                                            m->st.c));
    return DASH_OK;
}

dash_status recompute_c(dash_model *m, const BatchDev &b, const void *X) {
    const bool f64in = m->cfg.input_dtype == DASH_F64;
    if (m->tsize == 8)
        return f64in ? launch_recompute_c<double, double>(m, b, X) : launch_recompute_c<float, double>(m, b, X);
    return f64in ? launch_recompute_c<double, float>(m, b, X) : launch_recompute_c<float, float>(m, b, X);
}

dash_status run_update_p(dash_model *m, const BatchDev &b, const void *X, double lam, bool begin_new) {
    const bool f64in = m->cfg.input_dtype == DASH_F64;
    if (m->tsize == 8) {
        return f64in ? launch_update_p<double, double>(m, b, X, lam, begin_new)
                     : launch_update_p<float, double>(m, b, X, lam, begin_new);
    }
    return f64in ? launch_update_p<double, float>(m, b, X, lam, begin_new)
                 : launch_update_p<float, float>(m, b, X, lam, begin_new);
}

}  // namespace dash
