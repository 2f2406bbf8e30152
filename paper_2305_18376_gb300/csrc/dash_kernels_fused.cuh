// Fused single-pass mode-P row kernel (mixed precision: FP32 products,
// double-float per-slice summaries).
//
// One persistent CTA per SM walks a list of tiles.  A tile is a run of
// consecutive segments, each the only segment of its slice in this update,
// with at most FU_TILE_MAX rows in total, so the CTA owns every new row of
// its slices and can finish them before moving on:
//
//   phase A   Y = X_tile Ṽ with Ṽ = V Γ⁺ (Γ = VᵀV), so that for slices whose
//             S_k is nonsingular U_k,new = Y S_k⁻¹ (Lemma 1, Eq. 11, with
//             S(SΓS)⁺ = Γ⁺S⁻¹);  ||X||² for the fitness.
//   epilogue  per slice (one warp): U_k,new written out; ΔD = UᵀU;
//             Δc = diag(Uᵀ X V) = diag(ΔD S Γ); c_k ← λc_k + Δc,
//             D_k ← λD_k + ΔD (Eqs. 15-16, double-float);
//             W(k,:) = c_kᵀ(Γ ∗ D_k)⁺ (Eq. 12) by an FP32 Cholesky factor
//             refined twice with double-float residuals (FP64 Jacobi
//             pseudo-inverse when the factor is not trustworthy);
//             G share S_k ΔD S_k (Eq. 21); Ũ = U S_k,new kept on chip.
//   phase B   the CTA's share of F_inc = Σ X_kᵀ U_k S_k,new (Eq. 20): the same
//             tile is streamed again (it is still in L2) and Xᵀ Ũ accumulated.
//
// X rows arrive through a ring of FU_NBUF shared-memory slots filled by 1-D
// bulk async copies (cp.async.bulk) that complete on mbarriers; every wait
// is bounded and reports a timeout instead of hanging.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "small_linalg.cuh"

namespace dash {

constexpr int FU_THREADS = 256;
constexpr int FU_WARPS = 8;
constexpr int FU_TILE_MAX = 256;     // rows per tile (and max rows of a fused slice)
constexpr int FU_NBUF = 3;           // ring slots
constexpr int FU_SLOT_BYTES = 32768; // bytes per ring slot
constexpr int FU_JG = 64;            // max columns per warp group: J <= 8·64
constexpr int FU_SUB = 16;           // rows per phase-A reduction step
constexpr int FU_RP = 32;            // lanes = rank slots (R <= 32)
constexpr int FU_LD = 33;            // leading dimension of the per-warp R×R FP32 factor

struct FusedArgs {
    const float *X;
    int J, R;
    double lam, rtol;
    const float *Vt;          // Ṽ = V Γ⁺ (J×R)
    const df *Gdf;            // Γ (R×R) double-float
    const double *Gam;        // Γ (R×R) FP64
    const int *gam_ok;
    int n_tiles;
    const int *tile_s0, *tile_s1;  // segments [s0, s1) of each tile
    const int64_t *seg_row;
    const int *seg_slice;
    double *W;                // K×R
    df *c;                    // K×R
    df *D;                    // K×R×R
    float *U;                 // N×R output rows
    float *Fslot;             // gridDim × J×R partials of F_inc
    double *Gpart;            // gridDim × R×R partials of G_inc
    double *xn_part;          // gridDim partials of ||X||²
    double *wsp;              // per-warp FP64 workspace for the fallback paths
    int *err;                 // [0] wait timeouts, [1] fallback solves (count)
};

__host__ __device__ inline int fu_chunk_rows(int J) {
    int ch = FU_SLOT_BYTES / (J * 4);
    if (ch > 64) ch = 64;
    if (ch < 1) ch = 1;
    return ch;
}

__host__ __device__ inline size_t fu_wsp_doubles(int R) {
    return (size_t)4 * R * (R + 1) + 4 * (R + 1);
}

// shared memory layout (bytes)
__host__ __device__ inline size_t fu_smem_bytes(int J) {
    const int ch = fu_chunk_rows(J);
    size_t b = (size_t)FU_NBUF * ch * J * 4;               // ring
    b += (size_t)FU_WARPS * FU_SUB * FU_RP * 4;             // Ypart
    b += (size_t)FU_TILE_MAX * FU_RP * 4;                   // Ytile
    b += (size_t)FU_RP * FU_RP * 8;                         // Γ double-float
    b += (size_t)FU_WARPS * FU_RP * FU_LD * 4;              // per-warp FP32 factor
    b += (size_t)FU_WARPS * FU_RP * 8 * 2;                  // per-warp x (df), misc
    b += (size_t)FU_WARPS * FU_RP * 4 * 2;                  // per-warp vectors
    b += 64;                                                // mbarriers
    return b;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global → this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase: gives up after ~2·10⁹ cycles (≈ 1 s)
// and reports the timeout instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) {
            atomicAdd(err, 1);
            return false;
        }
    }
    return true;
}

// ---- warp-level FP32 Cholesky on a shared R×R block (lower) ---------------
__device__ inline bool warp_cholesky_f(float *A, int n, int ld, float tol) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; ++j) {
        __syncwarp();
        const float d = A[j * ld + j];
        if (!(d > tol)) return false;
        const float l = sqrtf(d);
        const float inv = 1.0f / l;
        for (int i = j + 1 + lane; i < n; i += 32) A[i * ld + j] *= inv;
        __syncwarp();
        if (lane == 0) A[j * ld + j] = l;
        for (int i = j + 1 + lane; i < n; i += 32) {
            const float lij = A[i * ld + j];
            for (int k = j + 1; k <= i; ++k) A[i * ld + k] -= lij * A[k * ld + j];
        }
    }
    __syncwarp();
    return true;
}

// solve L Lᵀ x = b for one right-hand side held one entry per lane (lane < n)
__device__ inline float warp_cholesky_solve_f(const float *L, int n, int ld, float b,
                                              float *tmp) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < n) tmp[lane] = b;
    for (int j = 0; j < n; ++j) {
        __syncwarp();
        const float yj = tmp[j] / L[j * ld + j];
        __syncwarp();
        if (lane == j) tmp[j] = yj;
        if (lane > j && lane < n) tmp[lane] -= L[lane * ld + j] * yj;
    }
    for (int j = n - 1; j >= 0; --j) {
        __syncwarp();
        const float xj = tmp[j] / L[j * ld + j];
        __syncwarp();
        if (lane == j) tmp[j] = xj;
        if (lane < j) tmp[lane] -= L[j * ld + lane] * xj;
    }
    __syncwarp();
    return lane < n ? tmp[lane] : 0.f;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(FU_THREADS, 1) k_rows_fused(FusedArgs a) {
    extern __shared__ __align__(128) unsigned char fsm[];
    const int J = a.J, R = a.R;
    const int CH = fu_chunk_rows(J);
    float *ring = reinterpret_cast<float *>(fsm);
    float *Ypart = ring + (size_t)FU_NBUF * CH * J;
    float *Ytile = Ypart + FU_WARPS * FU_SUB * FU_RP;
    df *Gs = reinterpret_cast<df *>(Ytile + FU_TILE_MAX * FU_RP);
    float *Lw_all = reinterpret_cast<float *>(Gs + FU_RP * FU_RP);
    df *xw_all = reinterpret_cast<df *>(Lw_all + FU_WARPS * FU_RP * FU_LD);
    float *vw_all = reinterpret_cast<float *>(xw_all + FU_WARPS * FU_RP * 2);
    uint64_t *bars = reinterpret_cast<uint64_t *>(vw_all + FU_WARPS * FU_RP * 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *Lw = Lw_all + warp * FU_RP * FU_LD;
    df *xw = xw_all + warp * FU_RP * 2;
    float *vw = vw_all + warp * FU_RP * 2;
    double *wsp = a.wsp + (size_t)(blockIdx.x * FU_WARPS + warp) * fu_wsp_doubles(R);

    // columns of this warp's group (multiple of 4 so the float4 loads align)
    int JGs = (J + FU_WARPS - 1) / FU_WARPS;
    JGs = (JGs + 3) & ~3;
    const int jb = warp * JGs;
    const int jn = max(0, min(JGs, J - jb));

    // Ṽ slice in registers: v[q] = Ṽ[jb + q][lane]
    float v[FU_JG];
#pragma unroll
    for (int q = 0; q < FU_JG; ++q)
        v[q] = (q < jn && lane < R) ? a.Vt[(int64_t)(jb + q) * R + lane] : 0.f;
    for (int i = tid; i < R * R; i += FU_THREADS) Gs[(i / R) * FU_RP + (i % R)] = a.Gdf[i];
    // this CTA's F partial starts at zero
    float *Fs = a.Fslot + (size_t)blockIdx.x * J * R;
    for (int i = tid; i < J * R; i += FU_THREADS) Fs[i] = 0.f;
    if (tid == 0) {
        for (int b = 0; b < FU_NBUF; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool gam_ok = *a.gam_ok != 0;

    // ---- chunk stream: for each of my tiles, phase A chunks then phase B ----
    // producer cursor (thread 0 only)
    int p_tile = blockIdx.x, p_phase = 0, p_chunk = 0;
    auto tile_rows = [&](int t, int64_t &r0, int64_t &r1) {
        r0 = a.seg_row[a.tile_s0[t]];
        r1 = a.seg_row[a.tile_s1[t]];
    };
    uint32_t issued = 0;       // chunks issued so far (thread 0)
    auto issue_next = [&]() {  // thread 0: issue the next chunk of the stream
        while (p_tile < a.n_tiles) {
            int64_t r0, r1;
            tile_rows(p_tile, r0, r1);
            const int nch = (int)((r1 - r0 + CH - 1) / CH);
            if (p_chunk < nch) {
                const int64_t cr0 = r0 + (int64_t)p_chunk * CH;
                const int cn = (int)((r1 - cr0) < CH ? (r1 - cr0) : CH);
                const int slot = issued % FU_NBUF;
                const uint32_t bytes = (uint32_t)cn * J * 4;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bars[slot], bytes);
                bulk_g2s(ring + (size_t)slot * CH * J, a.X + cr0 * J, bytes, &bars[slot]);
                ++issued;
                ++p_chunk;
                return;
            }
            p_chunk = 0;
            if (p_phase == 0) p_phase = 1;
            else { p_phase = 0; p_tile += gridDim.x; }
        }
    };
    if (tid == 0)
        for (int b = 0; b < FU_NBUF; ++b) issue_next();

    uint32_t consumed = 0;
    float xn_f = 0.f;
    double xn_d = 0.0;
    float gacc[FU_RP];                 // lane's row of this warp's G partial
#pragma unroll
    for (int s = 0; s < FU_RP; ++s) gacc[s] = 0.f;
    bool aborted = false;

    for (int t = blockIdx.x; t < a.n_tiles && !aborted; t += gridDim.x) {
        int64_t r0, r1;
        tile_rows(t, r0, r1);
        const int nr = (int)(r1 - r0);
        const int nch = (nr + CH - 1) / CH;
        // ================= phase A: Y = X Ṽ ================================
        for (int cI = 0; cI < nch; ++cI) {
            const int slot = consumed % FU_NBUF;
            const bool got = mbar_wait_bounded(&bars[slot], (consumed / FU_NBUF) & 1, &a.err[0]);
            if (__syncthreads_or(!got)) {      // one decision for the whole CTA
                aborted = true;
                break;
            }
            const float *xs = ring + (size_t)slot * CH * J;
            const int cn = min(CH, nr - cI * CH);
            for (int sub = 0; sub < cn; sub += FU_SUB) {
                const int sn = min(FU_SUB, cn - sub);
                for (int i = 0; i < sn; ++i) {
                    const float *xr = xs + (size_t)(sub + i) * J + jb;
                    float acc = 0.f, sq = 0.f;
#pragma unroll
                    for (int q = 0; q < FU_JG; q += 4) {
                        if (q < jn) {
                            const float4 x4 = *reinterpret_cast<const float4 *>(xr + q);
                            acc = fmaf(x4.x, v[q], acc);
                            acc = fmaf(x4.y, v[q + 1], acc);
                            acc = fmaf(x4.z, v[q + 2], acc);
                            acc = fmaf(x4.w, v[q + 3], acc);
                            sq = fmaf(x4.x, x4.x, sq);
                            sq = fmaf(x4.y, x4.y, sq);
                            sq = fmaf(x4.z, x4.z, sq);
                            sq = fmaf(x4.w, x4.w, sq);
                        }
                    }
                    Ypart[(warp * FU_SUB + i) * FU_RP + lane] = acc;
                    if (lane == 0) xn_f += sq;
                }
                __syncthreads();
                for (int o = tid; o < sn * FU_RP; o += FU_THREADS) {
                    const int i = o / FU_RP, l = o % FU_RP;
                    float s = 0.f;
#pragma unroll
                    for (int w = 0; w < FU_WARPS; ++w) s += Ypart[(w * FU_SUB + i) * FU_RP + l];
                    Ytile[(cI * CH + sub + i) * FU_RP + l] = s;
                }
                __syncthreads();
            }
            ++consumed;
            if (tid == 0) issue_next();
        }
        if (aborted) break;
        xn_d += (double)xn_f;
        xn_f = 0.f;
        // ================= epilogue: one warp per slice ======================
        const int s0 = a.tile_s0[t], s1 = a.tile_s1[t];
        for (int sg = s0 + warp; sg < s1; sg += FU_WARPS) {
            const int k = a.seg_slice[sg];
            const int ia = (int)(a.seg_row[sg] - r0);
            const int n = (int)(a.seg_row[sg + 1] - a.seg_row[sg]);
            const double wold_d = lane < R ? a.W[(int64_t)k * R + lane] : 1.0;
            const float wold = (float)wold_d;
            const bool fast = gam_ok && __all_sync(0xffffffffu, wold_d != 0.0);
            float dc = 0.f;                       // Δc[lane]
            if (fast) {
                const float winv = lane < R ? 1.0f / wold : 0.f;
                for (int i = 0; i < n; ++i) {
                    float *y = Ytile + (ia + i) * FU_RP;
                    const float u = y[lane] * winv;
                    __syncwarp();
                    y[lane] = u;
                    if (lane < R) a.U[(r0 + ia + i) * R + lane] = u;
                }
            } else {
                // general Lemma 1 map M = S (S Γ S)⁺ (FP64, rare): P = Y Γ, U = P M
                double *Aw = wsp, *Ew = Aw + R * (R + 1), *Mw = Ew + R * (R + 1);
                double *fw = Mw + R * (R + 1);
                const int ld = R + 1;
                for (int e = lane; e < R * R; e += 32) {
                    const int r = e / R, q = e % R;
                    Aw[r * ld + q] = a.W[(int64_t)k * R + r] * a.Gam[e] * a.W[(int64_t)k * R + q];
                }
                __syncwarp();
                warp_psd_pinv(Aw, Ew, fw, Mw, R, ld, a.rtol, 1, false);
                for (int e = lane; e < R * R; e += 32) {
                    const int r = e / R, q = e % R;
                    Mw[r * ld + q] *= a.W[(int64_t)k * R + r];
                }
                __syncwarp();
                for (int i = 0; i < n; ++i) {
                    float *y = Ytile + (ia + i) * FU_RP;
                    float p = 0.f;                            // P[i][lane] = Σ_t Y[i][t] Γ[t][lane]
                    for (int q = 0; q < R; ++q)
                        p = fmaf(y[q], lane < R ? Gs[q * FU_RP + lane].hi : 0.f, p);
                    float u = 0.f;                            // U[i][lane] = Σ_s P[i][s] M[s][lane]
                    for (int q = 0; q < R; ++q) {
                        const float ps = __shfl_sync(0xffffffffu, p, q);
                        if (lane < R) u = fmaf(ps, (float)Mw[q * ld + lane], u);
                    }
                    dc = fmaf(u, p, dc);
                    __syncwarp();
                    y[lane] = lane < R ? u : 0.f;
                    if (lane < R) a.U[(r0 + ia + i) * R + lane] = u;
                }
                atomicAdd(&a.err[1], 1);
            }
            __syncwarp();
            // ΔD row `lane`: dd[q] = Σ_i U[i][lane] U[i][q]
            float dd[FU_RP];
#pragma unroll
            for (int q = 0; q < FU_RP; ++q) dd[q] = 0.f;
            for (int i = 0; i < n; ++i) {
                const float *y = Ytile + (ia + i) * FU_RP;
                const float ul = y[lane];
#pragma unroll
                for (int q = 0; q < FU_RP; q += 4) {
                    const float4 y4 = *reinterpret_cast<const float4 *>(y + q);
                    dd[q] = fmaf(ul, y4.x, dd[q]);
                    dd[q + 1] = fmaf(ul, y4.y, dd[q + 1]);
                    dd[q + 2] = fmaf(ul, y4.z, dd[q + 2]);
                    dd[q + 3] = fmaf(ul, y4.w, dd[q + 3]);
                }
            }
            if (fast) {            // Δc = diag(ΔD S Γ): Δc[r] = Σ_q ΔD[r][q] w_q Γ[q][r]
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < FU_RP; ++q) {
                    const float wq = __shfl_sync(0xffffffffu, wold, q);
                    if (q < R && lane < R) s = fmaf(dd[q] * wq, Gs[q * FU_RP + lane].hi, s);
                }
                dc = s;
            }
            // c_k, D_k with λ (double-float), A = Γ ∗ D_k into the FP32 factor
            df cnew = {0.f, 0.f};
            float amax = 0.f;
            const float lamf_hi = (float)a.lam;
            const df lamdf = df_from_double(a.lam);
            df *Dk = a.D + (int64_t)k * R * R;
            if (lane < R) {
                const df cold = a.c[(int64_t)k * R + lane];
                cnew = df_add(a.lam == 0.0 ? df{0.f, 0.f} : df_mul(lamdf, cold), df_make(dc));
                a.c[(int64_t)k * R + lane] = cnew;
                for (int q = 0; q < R; ++q) {
                    const df dold = Dk[lane * R + q];
                    const df dn = df_add(a.lam == 0.0 ? df{0.f, 0.f} : df_mul(lamdf, dold),
                                         df_make(dd[q]));
                    Dk[lane * R + q] = dn;
                    const df av = df_mul(Gs[lane * FU_RP + q], dn);
                    Lw[lane * FU_LD + q] = av.hi;
                    if (q == lane) amax = fabsf(av.hi);
                }
            }
            (void)lamf_hi;
            amax = warp_max_f(amax);
            __syncwarp();
            // FP32 Cholesky, then two double-float refinement steps
            bool ok = amax > 0.f && warp_cholesky_f(Lw, R, FU_LD, 1e-6f * amax);
            df x = {0.f, 0.f};
            if (ok) {
                float x0 = warp_cholesky_solve_f(Lw, R, FU_LD, lane < R ? cnew.hi : 0.f, vw);
                x = df_make(x0);
                for (int it = 0; it < 2; ++it) {
                    __syncwarp();
                    if (lane < R) xw[lane] = x;
                    __syncwarp();
                    df res = cnew;
                    if (lane < R) {
                        for (int q = 0; q < R; ++q) {
                            const df av = df_mul(Gs[lane * FU_RP + q], Dk[lane * R + q]);
                            res = df_add(res, df_neg(df_mul(av, xw[q])));
                        }
                    }
                    const float dx = warp_cholesky_solve_f(Lw, R, FU_LD, lane < R ? res.hi : 0.f, vw);
                    x = df_add(x, df_make(dx));
                }
                // accept only if finite
                ok = __all_sync(0xffffffffu, isfinite(x.hi));
            }
            double wnew_d;
            if (ok) {
                wnew_d = lane < R ? df_to_double(x) : 0.0;
            } else {
                // FP64 pseudo-inverse solve (rare): A = Γ ∗ D_k, b = c_k
                double *Aw = wsp, *Lf = Aw + R * (R + 1), *Ew = Lf + R * (R + 1);
                double *bw = Ew + R * (R + 1), *fw = bw + (R + 1);
                const int ld = R + 1;
                __syncwarp();
                for (int e = lane; e < R * R; e += 32) {
                    const int r = e / R, q = e % R;
                    Aw[r * ld + q] = a.Gam[e] * df_to_double(Dk[e]);
                }
                if (lane < R) bw[lane] = df_to_double(cnew);
                __syncwarp();
                warp_psd_solve(Aw, Lf, Ew, bw, fw, R, ld, a.rtol);
                __syncwarp();
                wnew_d = lane < R ? bw[lane] : 0.0;
                atomicAdd(&a.err[1], 1);
            }
            if (lane < R) a.W[(int64_t)k * R + lane] = wnew_d;
            const float wnew = (float)wnew_d;
            // G share with the new S_k (Eq. 21): G[lane][q] += w_lane ΔD[lane][q] w_q
#pragma unroll
            for (int q = 0; q < FU_RP; ++q) {
                const float wq = __shfl_sync(0xffffffffu, wnew, q);
                if (lane < R && q < R) gacc[q] = fmaf(wnew * dd[q], wq, gacc[q]);
            }
            // Ũ = U S_k,new for phase B
            for (int i = 0; i < n; ++i) Ytile[(ia + i) * FU_RP + lane] *= (lane < R ? wnew : 0.f);
            __syncwarp();
        }
        __syncthreads();
        // ================= phase B: F partial += Xᵀ Ũ ========================
        float facc[FU_JG];
#pragma unroll
        for (int q = 0; q < FU_JG; ++q) facc[q] = 0.f;
        for (int cI = 0; cI < nch; ++cI) {
            const int slot = consumed % FU_NBUF;
            const bool got = mbar_wait_bounded(&bars[slot], (consumed / FU_NBUF) & 1, &a.err[0]);
            if (__syncthreads_or(!got)) {
                aborted = true;
                break;
            }
            const float *xs = ring + (size_t)slot * CH * J;
            const int cn = min(CH, nr - cI * CH);
            for (int i = 0; i < cn; ++i) {
                const float ut = Ytile[(cI * CH + i) * FU_RP + lane];
                const float *xr = xs + (size_t)i * J + jb;
#pragma unroll
                for (int q = 0; q < FU_JG; q += 4) {
                    if (q < jn) {
                        const float4 x4 = *reinterpret_cast<const float4 *>(xr + q);
                        facc[q] = fmaf(x4.x, ut, facc[q]);
                        facc[q + 1] = fmaf(x4.y, ut, facc[q + 1]);
                        facc[q + 2] = fmaf(x4.z, ut, facc[q + 2]);
                        facc[q + 3] = fmaf(x4.w, ut, facc[q + 3]);
                    }
                }
            }
            __syncthreads();
            ++consumed;
            if (tid == 0) issue_next();
        }
        if (aborted) break;
        if (lane < R) {
#pragma unroll
            for (int q = 0; q < FU_JG; ++q)
                if (q < jn) Fs[(int64_t)(jb + q) * R + lane] += facc[q];
        }
        __syncthreads();
    }
    if (aborted) {
        // let copies already issued land (bounded) before the CTA exits
        if (tid == 0) {
            for (uint32_t c = consumed; c < issued; ++c)
                mbar_wait_bounded(&bars[c % FU_NBUF], (c / FU_NBUF) & 1, &a.err[0]);
        }
        __syncthreads();
        return;
    }
    // ---- CTA partials of G and ||X||² (fixed order) -------------------------
    __syncthreads();
    float *gsm = Ypart;        // reuse: FU_WARPS × R × R floats (needs R*R*8 <= Ypart size)
    for (int q = 0; q < FU_RP; ++q)
        if (lane < R && q < R) gsm[(warp * FU_RP + lane) * FU_RP + q] = gacc[q];
    __syncthreads();
    for (int e = tid; e < R * R; e += FU_THREADS) {
        const int r = e / R, q = e % R;
        double s = 0.0;
        for (int w = 0; w < FU_WARPS; ++w) s += (double)gsm[(w * FU_RP + r) * FU_RP + q];
        a.Gpart[(int64_t)blockIdx.x * R * R + e] = s;
    }
    // ||X||²: lane 0 of each warp holds its warp's share
    __syncthreads();
    double *xsm = reinterpret_cast<double *>(Ytile);
    if (lane == 0) xsm[warp] = xn_d;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < FU_WARPS; ++w) s += xsm[w];
        a.xn_part[blockIdx.x] = s;
    }
}

// Ṽ = V Γ⁺ (FP32) and Γ in double-float, one warp per row of V.
__global__ void k_vtilde(const double *__restrict__ V, const double *__restrict__ GamP,
                         const double *__restrict__ Gam, int J, int R, float *__restrict__ Vt,
                         df *__restrict__ Gdf) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j < J) {
        for (int q = lane; q < R; q += 32) {
            double s = 0.0;
            for (int r = 0; r < R; ++r) s += V[(int64_t)j * R + r] * GamP[r * R + q];
            Vt[(int64_t)j * R + q] = (float)s;
        }
    }
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) Gdf[e] = df_from_double(Gam[e]);
}

}  // namespace dash
