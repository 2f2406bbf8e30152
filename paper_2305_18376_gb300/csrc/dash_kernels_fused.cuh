// Fused single-pass mode-P row kernel (mixed precision: FP32 products,
// double-float per-slice summaries).
//
// One persistent CTA per SM walks a list of tiles.  A tile is a run of
// consecutive segments, each the only segment of its slice in this update,
// with at most FU_TILE_MAX rows in total, so the CTA owns every new row of
// its slices and can finish them before moving on:
//
//   phase A   P' = X_tile Q_V with V = Q_V R_V (Q_V orthonormal): Theorem 1's
//             dominant product on a well-scaled operand; ||X||².
//   epilogue  per slice (one warp): U_k,new = X V S_k (S_k Γ S_k)⁻¹
//             = P' R_V⁻ᵀ S_k⁻¹ (Lemma 1, Eq. 11; Γ = VᵀV = R_VᵀR_V), which
//             loses digits to cond(V) only, not cond(V)²; the general map
//             S(SΓS)⁺ when S_k has zero entries; written out; ΔD = UᵀU;
//             Δc = diag(Uᵀ X V) = diag(ΔD S_k Γ) (X V = U S_k Γ);
//             c_k ← λc_k + Δc,
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "small_linalg.cuh"

namespace dash {

constexpr int FU_THREADS = 256;
constexpr int FU_WARPS = 8;
constexpr int kBigCBlocksPerSM = 3;   // CTAs per SM of k_big_c (and slots of the FP64 workspace)
constexpr int FU_TILE_MAX = 256;     // rows per tile (and max rows of a fused slice)
constexpr int FU_NBUF = 3;           // ring slots
constexpr int FU_SLOT_BYTES = 32768; // bytes per ring slot
constexpr int FU_JG = 64;            // max columns per warp group: J <= 8·64
constexpr int FU_SUB = 16;           // rows per phase-A reduction step
constexpr int FU_RP = 32;            // lanes = rank slots (R <= 32)
constexpr int FU_LD = 33;            // leading dimension of the per-warp R×R FP32 factor
constexpr int FU_YP = 36;            // pitch of the tile's Y / Ũ rows (conflict-free fragments)

// Ring rows are copied one by one into rows of pitch J + 8 floats, which keeps
// the 64-bit fragment loads of X conflict-free.
__host__ __device__ inline int fu_pitch(int J) { return J + 8; }

struct FusedArgs {
    const float *X;
    int J, R;
    double lam, rtol;
    float lam_hi, lam_lo;     // λ as double-float (lam_hi + lam_lo)
    int lam_on;               // λ != 0: the old summaries are kept
    const float *V32;         // Q_V (J×R, FP32): V = Q_V R_V with orthonormal Q_V
    const float *GPf;         // R_V⁻ᵀ (R×R, FP32, lower triangular)
    const double *RV;         // R_V (R×R, FP64, upper triangular)
    const df *Gdf;            // Γ (R×R) double-float
    const double *Gam;        // Γ (R×R) FP64
    const int *gam_ok;
    int n_tiles;
    const int *tile_s0, *tile_s1;  // segments [s0, s1) of each tile
    const int64_t *seg_row;
    const int *seg_slice;
    double *W;                // K×R
    float *Wf;                // K×R FP32 copy of the new weights (optional)
    df *c;                    // K×R
    df *D;                    // K×R×R
    float *U;                 // N×R output rows
    float *Fslot;             // gridDim × J×R partials of F_inc
    double *Gpart;            // gridDim × R×R partials of G_inc
    double *xn_part;          // gridDim partials of ||X||²
    double *wsp;              // per-warp FP64 workspace for the fallback paths
    int *err;                 // [0] wait timeouts, [1] fallback solves (count)
    unsigned long long *phase_cycles;  // optional: SM cycles in phase A, epilogue, phase B
};

__host__ __device__ inline int fu_chunk_rows(int J) {
    (void)J;
    return 16;                       // one 16-row MMA tile per chunk
}

__host__ __device__ inline size_t fu_wsp_doubles(int R) {
    return (size_t)4 * R * (R + 1) + 4 * (R + 1);
}

// shared memory layout (bytes)
__host__ __device__ inline size_t fu_smem_bytes(int J) {
    const int ch = fu_chunk_rows(J);
    size_t b = (size_t)FU_NBUF * ch * fu_pitch(J) * 4;      // ring
    b += (size_t)FU_WARPS * FU_SUB * FU_RP * 4;             // Ypart
    b += (size_t)FU_TILE_MAX * FU_YP * 4;                   // Ytile
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
// and reports the timeout instead of hanging: err[0] counts timeouts, err[3]
// marks the update as abandoned.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) {
            atomicAdd(err, 1);
            err[3] = 1;
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
        // trailing update of the lower triangle, one (i, k) pair per lane at a
        // time: m = n-j-1 remaining rows, pairs (a, b) with 0 <= b <= a < m
        const int m = n - j - 1;
        const int np = m * (m + 1) / 2;
        for (int p = lane; p < np; p += 32) {
            // row a of the pair index p: a(a+1)/2 <= p < (a+1)(a+2)/2
            int aa = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
            while ((aa + 1) * (aa + 2) / 2 <= p) ++aa;
            while (aa * (aa + 1) / 2 > p) --aa;
            const int bb = p - aa * (aa + 1) / 2;
            const int i = j + 1 + aa, k = j + 1 + bb;
            A[i * ld + k] -= A[i * ld + j] * A[k * ld + j];
        }
    }
    __syncwarp();
    return true;
}

// solve L Lᵀ x = b for one right-hand side held one entry per lane (lane < n);
// rinv holds 1/diag(L) (one entry per lane).  Lane i keeps its own entry in a
// register; the pivot of step j is broadcast with a shuffle.
__device__ inline float warp_cholesky_solve_f(const float *L, int n, int ld, float b,
                                              float rinv) {
    const int lane = threadIdx.x & 31;
    float y = lane < n ? b : 0.f;
    for (int j = 0; j < n; ++j) {
        const float yj = __shfl_sync(0xffffffffu, y * rinv, j);
        if (lane == j) y = yj;
        else if (lane > j && lane < n) y = fmaf(-L[lane * ld + j], yj, y);
    }
    for (int j = n - 1; j >= 0; --j) {
        const float xj = __shfl_sync(0xffffffffu, y * rinv, j);
        if (lane == j) y = xj;
        else if (lane < j) y = fmaf(-L[j * ld + lane], xj, y);
    }
    return lane < n ? y : 0.f;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// L Lᵀ x = b with lane i holding row i of L in `row` (registers) and L also
// in Lw (row i at Lw[i·FU_LD]); myinv = 1/L[i][i] on lane i.  Forward
// substitution broadcasts y_j from lane j; backward reads column entries
// L[j][i] from Lw.  Returns x[lane] (0 for lanes >= R).
__device__ __forceinline__ float chol_solve_reg(const float (&row)[FU_RP], const float *Lw,
                                                float myinv, bool act, float b) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float y = act ? b : 0.f;
#pragma unroll 32
    for (int j = 0; j < FU_RP; ++j) {
        const float yj = __shfl_sync(full, y * myinv, j);
        if (lane == j) y = yj;
        else if (lane > j) y = fmaf(-row[j], yj, y);
    }
#pragma unroll 32
    for (int j = FU_RP - 1; j >= 0; --j) {
        const float xj = __shfl_sync(full, y * myinv, j);
        if (lane == j) y = xj;
        else if (lane < j) y = fmaf(-Lw[j * FU_LD + lane], xj, y);
    }
    return act ? y : 0.f;
}

// Finish slice k from its new-data Gram ΔD (lane r holds row r in dd) and
// Δc (lane r holds Δc[r]): c_k ← λc_k + Δc, D_k ← λD_k + ΔD (Eqs. 15-16,
// double-float), W(k,:) = c_kᵀ(Γ ∗ D_k)⁺ (Eq. 12) by an FP32 Cholesky factor
// with one double-float refinement step (FP64 pseudo-inverse fallback), the
// slice's share S_k ΔD S_k of G_inc (Eq. 21) added to gacc (lane r: row r).
// Returns w_k,new[lane].  Called by all 32 lanes of a warp.
//
// Everything lives in registers, lane l owning row l: D_k is read and written
// column by column (coalesced; D_k is symmetric, so lane l's column is its
// row), A = Γ ∗ D_k is kept as double-float pairs, and the Cholesky factor is
// formed right-looking with the pivot column broadcast by shuffles.  Lw (a
// per-warp R×FU_LD float block) only carries L for the backward solve.
__device__ __forceinline__ float slice_finish(const FusedArgs &a, int k, const float (&dd)[FU_RP],
                                              float dc, float (&gacc)[FU_RP], const df *Gs,
                                              float *Lw, df *xw, double *wsp) {
    (void)xw;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int R = a.R;
    const bool act = lane < R;
    df cnew = {0.f, 0.f};
    const df lamdf = df_from_double(a.lam);
    const bool keep_old = a.lam != 0.0;
    df *Dk = a.D + (int64_t)k * R * R;
    if (act) {
        const df cold = a.c[(int64_t)k * R + lane];
        cnew = df_add(keep_old ? df_mul(lamdf, cold) : df{0.f, 0.f}, df_make(dc));
        a.c[(int64_t)k * R + lane] = cnew;
    }
    // D_k ← λD_k + ΔD and A = Γ ∗ D_k (row `lane`), coalesced over columns.
    // Rows and columns >= R stay zero: the factorisation below then runs over
    // all 32 (unrolled, no per-step guards) and leaves them zero.
    // (loads in batches of 4 ahead of the stores, so a batch costs one memory
    // round trip)
    float row[FU_RP];
    float mydiag = 0.f;
#pragma unroll
    for (int r0 = 0; r0 < FU_RP; r0 += 4) {
        df dold[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            dold[u] = (r0 + u < R && act && keep_old) ? Dk[(r0 + u) * R + lane] : df{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u;
            row[r] = 0.f;
            if (r < R && act) {
                const df dn = df_add(keep_old ? df_mul(lamdf, dold[u]) : df{0.f, 0.f}, df_make(dd[r]));
                Dk[r * R + lane] = dn;
                row[r] = df_mul(Gs[r * FU_RP + lane], dn).hi;      // Γ symmetric: conflict-free
                if (r == lane) mydiag = row[r];
            }
        }
    }
    const float amax = warp_max_f(fabsf(mydiag));
    // right-looking Cholesky of A (hi parts), lane l = row l
    const float tol = 1e-6f * amax;
    bool ok = amax > 0.f;
    float myinv = 0.f;
#pragma unroll 32
    for (int j = 0; j < FU_RP; ++j) {
        const float piv = __shfl_sync(full, row[j], j);
        if (j < R) ok = ok && (piv > tol);
        const float inv = rsqrtf(fmaxf(piv, 1e-30f));
        const float lij = (lane == j) ? piv * inv : row[j] * inv;
        row[j] = lij;
        if (lane == j) myinv = inv;
#pragma unroll 31
        for (int q = j + 1; q < FU_RP; ++q) {
            const float lqj = __shfl_sync(full, lij, q);
            row[q] = fmaf(-lij, lqj, row[q]);
        }
    }
    df x = {0.f, 0.f};
    if (ok) {
        // L (lower) to shared for the backward solve: Lw[i][j], row i by lane i
        __syncwarp();
#pragma unroll
        for (int j = 0; j < FU_RP; ++j) Lw[lane * FU_LD + j] = row[j];
        __syncwarp();
        const float x0 = chol_solve_reg(row, Lw, myinv, act, cnew.hi);
        // one refinement step: res = c − A x0 in double-float, A re-formed
        // from the D_k just written (an L1 hit)
        df res = cnew;
#pragma unroll
        for (int r = 0; r < FU_RP; ++r) {
            const float xr = __shfl_sync(full, x0, r);
            if (r < R && act) {
                const df av = df_mul(Gs[r * FU_RP + lane], Dk[r * R + lane]);
                res = df_sub(res, df_mul_f(av, xr));
            }
        }
        const float dx = chol_solve_reg(row, Lw, myinv, act, res.hi);
        x = df_add(df_make(x0), df_make(dx));
        ok = __all_sync(full, isfinite(x.hi));
    }
    double wnew_d;
    if (ok) {
        wnew_d = act ? df_to_double(x) : 0.0;
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
        if (act) bw[lane] = df_to_double(cnew);
        __syncwarp();
        warp_psd_solve(Aw, Lf, Ew, bw, fw, R, ld, a.rtol);
        __syncwarp();
        wnew_d = act ? bw[lane] : 0.0;
        if (lane == 0) atomicAdd(&a.err[1], 1);
    }
    if (act) a.W[(int64_t)k * R + lane] = wnew_d;
    if (act && a.Wf) a.Wf[(int64_t)k * R + lane] = (float)wnew_d;
    if (act && !isfinite(wnew_d)) atomicAdd(a.err + 2, 1);   // reported as DASH_ENUMERIC
    const float wnew = (float)wnew_d;
#pragma unroll
    for (int q = 0; q < FU_RP; ++q) {
        const float wq = __shfl_sync(full, wnew, q);
        if (act && q < R) gacc[q] = fmaf(wnew * dd[q], wq, gacc[q]);
    }
    __syncwarp();
    return wnew;
}

// ---- split products on the warp-level tensor-core MMA ------------------------
// x = hi + lo with hi = round(x), lo = round(x − hi) in FP16; a product a·b
// is taken as a_hi·b_hi + a_hi·b_lo + a_lo·b_hi (the error-corrected tensor
// core product of Ootomo and Yokota, 2022), accumulated in FP32.  FP16 halves carry ~22 significant bits per operand once it is scaled
// by a power of two so that its largest entries lie in [512, 1024) (per row
// and warp for X in P' = X Q_V, per tile for X and Ũ in the F sums, a fixed
// 2^9 for the orthonormal Q_V): the lo halves then stay in FP16's normal range
// and the MMA accumulates the exact products in FP32.
__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);   // x0 in the low half
    const float2 hf = __bfloat1622float2(h);
    hi = bf16x2_bits(h);
    lo = bf16x2_bits(__floats2bfloat162_rn(x0 - hf.x, x1 - hf.y));
}
// FP16 split: 11-bit mantissas, so hi + lo carries ~22 bits when both halves
// are normal numbers; callers scale operands by powers of two first.
__device__ __forceinline__ uint32_t half2_bits(__half2 v) { return *reinterpret_cast<uint32_t *>(&v); }
// lo is stored scaled by 2^11 so that it stays a normal FP16 number; the
// correction products are scaled back by 2^-11 after the MMA.
__device__ __forceinline__ void split_pair_h(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    hi = half2_bits(h);
    lo = half2_bits(__floats2half2_rn((x0 - hf.x) * 2048.f, (x1 - hf.y) * 2048.f));
}
__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                        uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// acc += a_hi·b_hi + 2^-11 (a_hi·b_lo' + a_lo'·b_hi) for one 16×8×16 tile, with
// the main and correction products accumulated separately from zero inside
// the tensor core and added to acc with IEEE FP32 adds (the tensor core's
// own FP32 accumulation truncates when aligning a small term to a large one).
__device__ __forceinline__ void mma_split3(float (&acc)[4], const uint32_t (&ah)[4],
                                           const uint32_t (&al)[4], uint32_t bh0, uint32_t bh1,
                                           uint32_t bl0, uint32_t bl1) {
    float dm[4] = {0.f, 0.f, 0.f, 0.f}, dc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_f16(dm, ah, bh0, bh1);
    mma_f16(dc, ah, bl0, bl1);
    mma_f16(dc, al, bh0, bh1);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += fmaf(dc[e], 4.8828125e-4f, dm[e]);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// TC = true: phases A and B on tensor cores (BF16 split, 3 products);
// TC = false: FP32 CUDA-core FMAs.
template <bool TC>
__global__ void __launch_bounds__(FU_THREADS, 1) k_rows_fused(FusedArgs a) {
    extern __shared__ __align__(128) unsigned char fsm[];
    const int J = a.J, R = a.R;
    const int CH = fu_chunk_rows(J);
    const int P = fu_pitch(J);
    float *ring = reinterpret_cast<float *>(fsm);
    float *Ypart = ring + (size_t)FU_NBUF * CH * P;
    float *Ytile = Ypart + FU_WARPS * FU_SUB * FU_RP;
    df *Gs = reinterpret_cast<df *>(Ytile + FU_TILE_MAX * FU_YP);
    float *Lw_all = reinterpret_cast<float *>(Gs + FU_RP * FU_RP);
    df *xw_all = reinterpret_cast<df *>(Lw_all + FU_WARPS * FU_RP * FU_LD);
    float *vw_all = reinterpret_cast<float *>(xw_all + FU_WARPS * FU_RP * 2);
    uint64_t *bars = reinterpret_cast<uint64_t *>(vw_all + FU_WARPS * FU_RP * 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tg = lane & 3;        // MMA fragment coordinates
    float *red = vw_all;                           // per-warp maxima for the tile scales
    float *Lw = Lw_all + warp * FU_RP * FU_LD;
    df *xw = xw_all + warp * FU_RP * 2;
    double *wsp = a.wsp + (size_t)(blockIdx.x * FU_WARPS + warp) * fu_wsp_doubles(R);

    // columns of this warp's group: multiples of 16 (TC) or 4 (float4 loads)
    int JGs = (J + FU_WARPS - 1) / FU_WARPS;
    JGs = TC ? ((JGs + 15) & ~15) : ((JGs + 3) & ~3);
    const int jb = warp * JGs;
    const int jn = max(0, min(JGs, J - jb));

    // V slice in registers.  SIMT: v[q] = V[jb + q][lane].  TC: B fragments
    // of V (k = j, n = r) for 4 k-steps × 4 n-tiles, hi and lo halves.
    float v[TC ? 1 : FU_JG];
    uint32_t vbh[TC ? 4 : 1][4][2], vbl[TC ? 4 : 1][4][2];
    if constexpr (!TC) {
#pragma unroll
        for (int q = 0; q < FU_JG; ++q)
            v[q] = (q < jn && lane < R) ? a.V32[(int64_t)(jb + q) * R + lane] : 0.f;
    } else {
#pragma unroll
        for (int st = 0; st < 4; ++st)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = jb + 16 * st + 8 * h + 2 * tg;
                    const int n = 8 * nt + g;
                    const bool ok0 = (16 * st + 8 * h + 2 * tg) < jn && n < R;
                    // |Q_V| <= 1: scaled by 2^9 so that the lo halves stay normal
                    const float v0 = ok0 ? a.V32[(int64_t)j * R + n] * 512.f : 0.f;
                    const float v1 = ok0 ? a.V32[(int64_t)(j + 1) * R + n] * 512.f : 0.f;
                    split_pair_h(v0, v1, vbh[st][nt][h], vbl[st][nt][h]);
                }
    }
    for (int i = tid; i < R * R; i += FU_THREADS) Gs[(i / R) * FU_RP + (i % R)] = a.Gdf[i];
    // this CTA's F partial starts at zero; so does the ring (its row padding is read)
    float *Fs = a.Fslot + (size_t)blockIdx.x * J * R;
    for (int i = tid; i < J * R; i += FU_THREADS) Fs[i] = 0.f;
    for (int i = tid; i < FU_NBUF * CH * P; i += FU_THREADS) ring[i] = 0.f;
    for (int i = tid; i < FU_TILE_MAX * FU_YP; i += FU_THREADS) Ytile[i] = 0.f;
    if (tid == 0) {
        for (int b = 0; b < FU_NBUF; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool gam_ok = *a.gam_ok != 0;

    // ---- chunk stream: for each of my tiles, phase A chunks then phase B ----
    int p_tile = blockIdx.x, p_phase = 0, p_chunk = 0;   // producer cursor (thread 0)
    auto tile_rows = [&](int t, int64_t &r0, int64_t &r1) {
        r0 = a.seg_row[a.tile_s0[t]];
        r1 = a.seg_row[a.tile_s1[t]];
    };
    uint32_t issued = 0;
    auto issue_next = [&]() {  // thread 0: copy the next chunk, row by row, into its slot
        while (p_tile < a.n_tiles) {
            int64_t r0, r1;
            tile_rows(p_tile, r0, r1);
            const int nch = (int)((r1 - r0 + CH - 1) / CH);
            if (p_chunk < nch) {
                const int64_t cr0 = r0 + (int64_t)p_chunk * CH;
                const int cn = (int)((r1 - cr0) < CH ? (r1 - cr0) : CH);
                const int slot = issued % FU_NBUF;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bars[slot], (uint32_t)cn * J * 4);
                float *dst = ring + (size_t)slot * CH * P;
                for (int r = 0; r < cn; ++r)
                    bulk_g2s(dst + (size_t)r * P, a.X + (cr0 + r) * J, (uint32_t)J * 4, &bars[slot]);
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
    for (int q = 0; q < FU_RP; ++q) gacc[q] = 0.f;
    bool aborted = false;
    unsigned long long cyc[3] = {0ull, 0ull, 0ull};
    long long wcyc[4] = {0, 0, 0, 0};      // per warp: U rows, ΔD, slice finish, Ũ scaling
    long long tmark = clock64();
    float xmax_t = 0.f;                // max |x| of the current tile (this thread's share)

    for (int t = blockIdx.x; t < a.n_tiles && !aborted; t += gridDim.x) {
        int64_t r0, r1;
        tile_rows(t, r0, r1);
        const int nr = (int)(r1 - r0);
        const int nch = (nr + CH - 1) / CH;
        {
            // bring this tile's per-slice state (D_k, c_k, W(k,:)) into L2 while
            // phase A streams X, so the epilogue does not wait on HBM for it
            const int ts0 = a.tile_s0[t], ts1 = a.tile_s1[t];
            const int ld_ = (R * R * 8 + 127) / 128, lc = (R * 8 + 127) / 128;
            const int per = ld_ + 2 * lc;
            for (int e = tid; e < (ts1 - ts0) * per; e += FU_THREADS) {
                const int k = a.seg_slice[ts0 + e / per], l = e % per;
                const char *pp;
                if (l < ld_) pp = reinterpret_cast<const char *>(a.D + (int64_t)k * R * R) + l * 128;
                else if (l < ld_ + lc) pp = reinterpret_cast<const char *>(a.c + (int64_t)k * R) + (l - ld_) * 128;
                else pp = reinterpret_cast<const char *>(a.W + (int64_t)k * R) + (l - ld_ - lc) * 128;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pp));
            }
        }
        // ================= phase A: P = X V =================================
        for (int cI = 0; cI < nch; ++cI) {
            const int slot = consumed % FU_NBUF;
            const bool got = mbar_wait_bounded(&bars[slot], (consumed / FU_NBUF) & 1, &a.err[0]);
            if (__syncthreads_or(!got)) {      // one decision for the whole CTA
                aborted = true;
                break;
            }
            const float *xs = ring + (size_t)slot * CH * P;
            const int cn = min(CH, nr - cI * CH);
            if constexpr (TC) {
                float yacc[4][4];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) yacc[nt][e] = 0.f;
                float2 xa_[4][4];
                float m0 = 0.f, m1 = 0.f;   // row maxima over this warp's columns
#pragma unroll
                for (int st = 0; st < 4; ++st) {
                    if (16 * st < jn) {
                        const int j0 = jb + 16 * st + 2 * tg;
                        const bool c0 = (16 * st + 2 * tg) < jn, c1 = (16 * st + 8 + 2 * tg) < jn;
                        const bool rg0 = g < cn, rg1 = g + 8 < cn;
                        const float2 z = make_float2(0.f, 0.f);
                        const float2 x00 = (rg0 && c0) ? *reinterpret_cast<const float2 *>(xs + g * P + j0) : z;
                        const float2 x10 = (rg1 && c0) ? *reinterpret_cast<const float2 *>(xs + (g + 8) * P + j0) : z;
                        const float2 x01 = (rg0 && c1) ? *reinterpret_cast<const float2 *>(xs + g * P + j0 + 8) : z;
                        const float2 x11 = (rg1 && c1) ? *reinterpret_cast<const float2 *>(xs + (g + 8) * P + j0 + 8) : z;
                        xn_f += x00.x * x00.x + x00.y * x00.y + x10.x * x10.x + x10.y * x10.y +
                                x01.x * x01.x + x01.y * x01.y + x11.x * x11.x + x11.y * x11.y;
                        xa_[st][0] = x00; xa_[st][1] = x10; xa_[st][2] = x01; xa_[st][3] = x11;
                        m0 = fmaxf(m0, fmaxf(fmaxf(fabsf(x00.x), fabsf(x00.y)), fmaxf(fabsf(x01.x), fabsf(x01.y))));
                        m1 = fmaxf(m1, fmaxf(fmaxf(fabsf(x10.x), fabsf(x10.y)), fmaxf(fabsf(x11.x), fabsf(x11.y))));
                    } else {
                        const float2 z = make_float2(0.f, 0.f);
                        xa_[st][0] = z; xa_[st][1] = z; xa_[st][2] = z; xa_[st][3] = z;
                    }
                }
                // power-of-two scale of rows g and g+8 over this warp's columns:
                // the four lanes of a row group share the row
                xmax_t = fmaxf(xmax_t, fmaxf(m0, m1));
                m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
                m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
                m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
                m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
                // rows scaled into [512, 1024): FP16 lo halves stay normal
                int e0 = 0, e1 = 0;
                if (m0 > 0.f) frexpf(m0, &e0);
                if (m1 > 0.f) frexpf(m1, &e1);
                const float s0 = ldexpf(1.f, 10 - e0), s1 = ldexpf(1.f, 10 - e1);
#pragma unroll
                for (int st = 0; st < 4; ++st) {
                    if (16 * st < jn) {
                        uint32_t ah[4], al[4];
                        split_pair_h(xa_[st][0].x * s0, xa_[st][0].y * s0, ah[0], al[0]);
                        split_pair_h(xa_[st][1].x * s1, xa_[st][1].y * s1, ah[1], al[1]);
                        split_pair_h(xa_[st][2].x * s0, xa_[st][2].y * s0, ah[2], al[2]);
                        split_pair_h(xa_[st][3].x * s1, xa_[st][3].y * s1, ah[3], al[3]);
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
                            mma_split3(yacc[nt], ah, al, vbh[st][nt][0], vbh[st][nt][1],
                                       vbl[st][nt][0], vbl[st][nt][1]);
                    }
                }
                const float u0 = ldexpf(1.f, e0 - 19), u1 = ldexpf(1.f, e1 - 19);   // 2^(e-10)·2^-9
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    yacc[nt][0] *= u0;
                    yacc[nt][1] *= u0;
                    yacc[nt][2] *= u1;
                    yacc[nt][3] *= u1;
                }
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int c = 8 * nt + 2 * tg;
                    *reinterpret_cast<float2 *>(&Ypart[(warp * FU_SUB + g) * FU_RP + c]) =
                        make_float2(yacc[nt][0], yacc[nt][1]);
                    *reinterpret_cast<float2 *>(&Ypart[(warp * FU_SUB + g + 8) * FU_RP + c]) =
                        make_float2(yacc[nt][2], yacc[nt][3]);
                }
                __syncthreads();
                for (int o = tid; o < cn * FU_RP; o += FU_THREADS) {
                    const int i = o / FU_RP, l = o % FU_RP;
                    float sacc = 0.f;
#pragma unroll
                    for (int w = 0; w < FU_WARPS; ++w) sacc += Ypart[(w * FU_SUB + i) * FU_RP + l];
                    Ytile[(cI * CH + i) * FU_YP + l] = sacc;
                }
                __syncthreads();
            } else {
                for (int sub = 0; sub < cn; sub += FU_SUB) {
                    const int sn = min(FU_SUB, cn - sub);
                    for (int i = 0; i < sn; ++i) {
                        const float *xr = xs + (size_t)(sub + i) * P + jb;
                        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, sq0 = 0.f, sq1 = 0.f;
#pragma unroll
                        for (int q = 0; q < FU_JG; q += 4) {
                            if (q < jn) {
                                const float4 x4 = *reinterpret_cast<const float4 *>(xr + q);
                                a0 = fmaf(x4.x, v[q], a0);
                                a1 = fmaf(x4.y, v[q + 1], a1);
                                a2 = fmaf(x4.z, v[q + 2], a2);
                                a3 = fmaf(x4.w, v[q + 3], a3);
                                sq0 = fmaf(x4.x, x4.x, sq0);
                                sq1 = fmaf(x4.y, x4.y, sq1);
                                sq0 = fmaf(x4.z, x4.z, sq0);
                                sq1 = fmaf(x4.w, x4.w, sq1);
                            }
                        }
                        Ypart[(warp * FU_SUB + i) * FU_RP + lane] = (a0 + a1) + (a2 + a3);
                        if (lane == 0) xn_f += sq0 + sq1;
                    }
                    __syncthreads();
                    for (int o = tid; o < sn * FU_RP; o += FU_THREADS) {
                        const int i = o / FU_RP, l = o % FU_RP;
                        float sacc = 0.f;
#pragma unroll
                        for (int w = 0; w < FU_WARPS; ++w) sacc += Ypart[(w * FU_SUB + i) * FU_RP + l];
                        Ytile[(cI * CH + sub + i) * FU_YP + l] = sacc;
                    }
                    __syncthreads();
                }
            }
            ++consumed;
            if (tid == 0) issue_next();
        }
        if (aborted) break;
        xn_d += (double)xn_f;
        xn_f = 0.f;
        {
            const long long now = clock64();
            cyc[0] += (unsigned long long)(now - tmark);
            tmark = now;
        }
        // ================= epilogue: one warp per slice ======================
        const int s0 = a.tile_s0[t], s1 = a.tile_s1[t];
        for (int sg = s0 + warp; sg < s1; sg += FU_WARPS) {
            long long w0 = a.phase_cycles ? clock64() : 0;
            const int k = a.seg_slice[sg];
            const int ia = (int)(a.seg_row[sg] - r0);
            const int n = (int)(a.seg_row[sg + 1] - a.seg_row[sg]);
            const double wold_d = lane < R ? a.W[(int64_t)k * R + lane] : 1.0;
            const float wold = (float)wold_d;
            const bool fast = gam_ok && __all_sync(0xffffffffu, wold_d != 0.0);
            float dc = 0.f;                       // Δc[lane]
            // U = P' mcol: fast path mcol = column `lane` of R_V⁻ᵀ S⁻¹; general
            // path (zero weights) mcol = column of R_V S (S Γ S)⁺ (FP64, rare)
            float mcol[FU_RP], rvcol[FU_RP];
            if (fast) {
                const float winv = lane < R ? 1.0f / wold : 0.f;
#pragma unroll
                for (int t = 0; t < FU_RP; ++t) {
                    mcol[t] = (t < R && lane < R) ? a.GPf[t * R + lane] * winv : 0.f;
                    rvcol[t] = 0.f;
                }
            } else {
                double *Aw = wsp, *Ew = Aw + R * (R + 1), *Mw = Ew + R * (R + 1);
                double *fw = Mw + R * (R + 1);
                const int ld = R + 1;
                for (int e = lane; e < R * R; e += 32) {
                    const int r = e / R, q = e % R;
                    Aw[r * ld + q] = a.W[(int64_t)k * R + r] * a.Gam[e] * a.W[(int64_t)k * R + q];
                }
                __syncwarp();
                warp_psd_pinv(Aw, Ew, fw, Mw, R, ld, a.rtol, 1, false);
                __syncwarp();
#pragma unroll
                for (int t = 0; t < FU_RP; ++t) {
                    double m = 0.0;
                    if (t < R && lane < R)
                        for (int q = t; q < R; ++q)
                            m += a.RV[t * R + q] * a.W[(int64_t)k * R + q] * Mw[q * ld + lane];
                    mcol[t] = (float)m;
                    rvcol[t] = (t < R && lane < R) ? (float)a.RV[t * R + lane] : 0.f;
                }
                if (lane == 0) atomicAdd(&a.err[1], 1);
            }
            for (int i = 0; i < n; ++i) {
                float *y = Ytile + (ia + i) * FU_YP;
                float u0 = 0.f, u1 = 0.f, pl = 0.f;
#pragma unroll
                for (int t = 0; t < FU_RP; t += 4) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(y + t);
                    u0 = fmaf(p4.x, mcol[t], u0);
                    u1 = fmaf(p4.y, mcol[t + 1], u1);
                    u0 = fmaf(p4.z, mcol[t + 2], u0);
                    u1 = fmaf(p4.w, mcol[t + 3], u1);
                }
                if (!fast) {                      // general path: Σ_i U(i,r) (X V)(i,r)
#pragma unroll
                    for (int t = 0; t < FU_RP; t += 4) {
                        const float4 p4 = *reinterpret_cast<const float4 *>(y + t);
                        pl = fmaf(p4.x, rvcol[t], pl);
                        pl = fmaf(p4.y, rvcol[t + 1], pl);
                        pl = fmaf(p4.z, rvcol[t + 2], pl);
                        pl = fmaf(p4.w, rvcol[t + 3], pl);
                    }
                }
                const float u = u0 + u1;
                dc = fmaf(u, pl, dc);
                __syncwarp();
                y[lane] = u;
                if (lane < R) a.U[(r0 + ia + i) * R + lane] = u;
            }
            __syncwarp();
            if (a.phase_cycles) { const long long w1 = clock64(); wcyc[0] += w1 - w0; w0 = w1; }
            // ΔD row `lane`: dd[q] = Σ_i U[i][lane] U[i][q]
            float dd[FU_RP];
#pragma unroll
            for (int q = 0; q < FU_RP; ++q) dd[q] = 0.f;
            for (int i = 0; i < n; ++i) {
                const float *y = Ytile + (ia + i) * FU_YP;
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
                float sacc = 0.f;
#pragma unroll
                for (int q = 0; q < FU_RP; ++q) {
                    const float wq = __shfl_sync(0xffffffffu, wold, q);
                    if (q < R && lane < R) sacc = fmaf(dd[q] * wq, Gs[q * FU_RP + lane].hi, sacc);
                }
                dc = sacc;
            }
            if (a.phase_cycles) { const long long w1 = clock64(); wcyc[1] += w1 - w0; w0 = w1; }
            const float wnew = slice_finish(a, k, dd, dc, gacc, Gs, Lw, xw, wsp);
            if (a.phase_cycles) { const long long w1 = clock64(); wcyc[2] += w1 - w0; w0 = w1; }
            // Ũ = U S_k,new for phase B
            for (int i = 0; i < n; ++i) Ytile[(ia + i) * FU_YP + lane] *= (lane < R ? wnew : 0.f);
            __syncwarp();
            if (a.phase_cycles) { const long long w1 = clock64(); wcyc[3] += w1 - w0; }
        }
        __syncthreads();
        {
            const long long now = clock64();
            cyc[1] += (unsigned long long)(now - tmark);
            tmark = now;
        }
        // ================= phase B: F partial += Xᵀ Ũ ========================
        float facc[TC ? 4 : 1][4][4];        // TC: m-tile (j) × n-tile (r) × fragment
        float fs[TC ? 1 : FU_JG];            // SIMT: one column r = lane, j = jb + q
        float sx = 1.f, su = 1.f;            // TC: power-of-two tile scales of X and Ũ
        int ex = 0, eu = 0;
        if constexpr (TC) {
            // tile maxima of |X| (from phase A) and |Ũ|, reduced over the CTA
            float um = 0.f;
            for (int o = tid; o < nr * FU_RP; o += FU_THREADS)
                um = fmaxf(um, fabsf(Ytile[(o / FU_RP) * FU_YP + (o % FU_RP)]));
            float xm = xmax_t;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, off));
                um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, off));
            }
            if (lane == 0) {
                red[warp] = xm;
                red[FU_WARPS + warp] = um;
            }
            __syncthreads();
            xm = 0.f;
            um = 0.f;
#pragma unroll
            for (int w = 0; w < FU_WARPS; ++w) {
                xm = fmaxf(xm, red[w]);
                um = fmaxf(um, red[FU_WARPS + w]);
            }
            if (xm > 0.f) frexpf(xm, &ex);
            if (um > 0.f) frexpf(um, &eu);
            ex -= 10;                        // scaled maxima in [512, 1024)
            eu -= 10;
            sx = ldexpf(1.f, -ex);
            su = ldexpf(1.f, -eu);
            xmax_t = 0.f;
            __syncthreads();
        }
        if constexpr (TC) {
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) facc[mt][nt][e] = 0.f;
        } else {
#pragma unroll
            for (int q = 0; q < FU_JG; ++q) fs[q] = 0.f;
        }
        for (int cI = 0; cI < nch; ++cI) {
            const int slot = consumed % FU_NBUF;
            const bool got = mbar_wait_bounded(&bars[slot], (consumed / FU_NBUF) & 1, &a.err[0]);
            if (__syncthreads_or(!got)) {
                aborted = true;
                break;
            }
            const float *xs = ring + (size_t)slot * CH * P;
            const int cn = min(CH, nr - cI * CH);
            if constexpr (TC) {
                // B fragments of Ũ (k = row, n = r): rows 2tg, 2tg+1 and +8
                const float *ut = Ytile + (size_t)(cI * CH) * FU_YP;
                const bool k0 = 2 * tg < cn, k1 = 2 * tg + 1 < cn, k2 = 2 * tg + 8 < cn, k3 = 2 * tg + 9 < cn;
                uint32_t bh[4][2], bl[4][2];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int c = 8 * nt + g;
                    split_pair_h(k0 ? ut[(2 * tg) * FU_YP + c] * su : 0.f,
                                 k1 ? ut[(2 * tg + 1) * FU_YP + c] * su : 0.f, bh[nt][0], bl[nt][0]);
                    split_pair_h(k2 ? ut[(2 * tg + 8) * FU_YP + c] * su : 0.f,
                                 k3 ? ut[(2 * tg + 9) * FU_YP + c] * su : 0.f, bh[nt][1], bl[nt][1]);
                }
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    if (16 * mt < jn) {
                        // A fragments of Xᵀ (m = j, k = row)
                        const int jm = jb + 16 * mt + g;
                        const bool m0 = (16 * mt + g) < jn, m1 = (16 * mt + g + 8) < jn;
                        float xa[8];
                        xa[0] = (m0 && k0) ? xs[(2 * tg) * P + jm] : 0.f;
                        xa[1] = (m0 && k1) ? xs[(2 * tg + 1) * P + jm] : 0.f;
                        xa[2] = (m1 && k0) ? xs[(2 * tg) * P + jm + 8] : 0.f;
                        xa[3] = (m1 && k1) ? xs[(2 * tg + 1) * P + jm + 8] : 0.f;
                        xa[4] = (m0 && k2) ? xs[(2 * tg + 8) * P + jm] : 0.f;
                        xa[5] = (m0 && k3) ? xs[(2 * tg + 9) * P + jm] : 0.f;
                        xa[6] = (m1 && k2) ? xs[(2 * tg + 8) * P + jm + 8] : 0.f;
                        xa[7] = (m1 && k3) ? xs[(2 * tg + 9) * P + jm + 8] : 0.f;
                        uint32_t ah[4], al[4];
                        split_pair_h(xa[0] * sx, xa[1] * sx, ah[0], al[0]);
                        split_pair_h(xa[2] * sx, xa[3] * sx, ah[1], al[1]);
                        split_pair_h(xa[4] * sx, xa[5] * sx, ah[2], al[2]);
                        split_pair_h(xa[6] * sx, xa[7] * sx, ah[3], al[3]);
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
                            mma_split3(facc[mt][nt], ah, al, bh[nt][0], bh[nt][1], bl[nt][0],
                                       bl[nt][1]);
                    }
                }
            } else {
                for (int i = 0; i < cn; ++i) {
                    const float ut = Ytile[(cI * CH + i) * FU_YP + lane];
                    const float *xr = xs + (size_t)i * P + jb;
#pragma unroll
                    for (int q = 0; q < FU_JG; q += 4) {
                        if (q < jn) {
                            const float4 x4 = *reinterpret_cast<const float4 *>(xr + q);
                            fs[q] = fmaf(x4.x, ut, fs[q]);
                            fs[q + 1] = fmaf(x4.y, ut, fs[q + 1]);
                            fs[q + 2] = fmaf(x4.z, ut, fs[q + 2]);
                            fs[q + 3] = fmaf(x4.w, ut, fs[q + 3]);
                        }
                    }
                }
            }
            __syncthreads();
            ++consumed;
            if (tid == 0) issue_next();
        }
        if (aborted) break;
        if constexpr (TC) {
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int jl = 16 * mt + g + 8 * (e >> 1);
                        const int r = 8 * nt + 2 * tg + (e & 1);
                        if (jl < jn && r < R)
                            Fs[(int64_t)(jb + jl) * R + r] += ldexpf(facc[mt][nt][e], ex + eu);
                    }
        } else {
            if (lane < R) {
#pragma unroll
                for (int q = 0; q < FU_JG; ++q)
                    if (q < jn) Fs[(int64_t)(jb + q) * R + lane] += fs[q];
            }
        }
        __syncthreads();
        {
            const long long now = clock64();
            cyc[2] += (unsigned long long)(now - tmark);
            tmark = now;
        }
    }
    if (a.phase_cycles && tid == 0) {
        atomicAdd(&a.phase_cycles[0], cyc[0]);
        atomicAdd(&a.phase_cycles[1], cyc[1]);
        atomicAdd(&a.phase_cycles[2], cyc[2]);
    }
    if (a.phase_cycles && lane == 0) {     // epilogue sub-phases, summed over warps
#pragma unroll
        for (int i = 0; i < 4; ++i) atomicAdd(&a.phase_cycles[3 + i], (unsigned long long)wcyc[i]);
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
    float *gsm = Ypart;        // FU_WARPS × FU_RP × FU_RP floats: spans Ypart and Ytile
#pragma unroll
    for (int q = 0; q < FU_RP; ++q) gsm[(warp * FU_RP + lane) * FU_RP + q] = gacc[q];
    __syncthreads();
    for (int e = tid; e < R * R; e += FU_THREADS) {
        const int r = e / R, q = e % R;
        double sacc = 0.0;
        for (int w = 0; w < FU_WARPS; ++w) sacc += (double)gsm[(w * FU_RP + r) * FU_RP + q];
        a.Gpart[(int64_t)blockIdx.x * R * R + e] = sacc;
    }
    __syncthreads();
    // ||X||²: TC — every lane holds a distinct share; SIMT — lane 0 of each warp
    double xs_d = TC ? (double)xn_d : (lane == 0 ? xn_d : 0.0);
    xs_d = warp_sum(xs_d);
    double *xsm = reinterpret_cast<double *>(Ytile + 2 * FU_WARPS * FU_RP);
    if (lane == 0) xsm[warp] = xs_d;
    __syncthreads();
    if (tid == 0) {
        double sacc = 0.0;
        for (int w = 0; w < FU_WARPS; ++w) sacc += xsm[w];
        a.xn_part[blockIdx.x] = sacc;
    }
}

// V = Q_V R_V from Γ = VᵀV = R_VᵀR_V (Cholesky, FP64, one warp): R_V (upper),
// L⁻¹ = R_V⁻ᵀ (lower) in FP64 and FP32, and Γ in double-float.  Sets *gam_ok
// to whether Γ is safely positive definite (the same test as Γ⁺).
static __global__ void k_vqr(const double *__restrict__ Gam, int R, double rtol, double *__restrict__ RV,
                      double *__restrict__ Linv, float *__restrict__ LinvF, df *__restrict__ Gdf,
                      int *__restrict__ gam_ok) {
    extern __shared__ double qsm[];
    const int ld = R + 1, lane = threadIdx.x & 31;
    double *L = qsm, *Li = qsm + R * ld, *rinv = Li + R * ld;
    for (int e = lane; e < R * R; e += 32) {
        L[(e / R) * ld + (e % R)] = Gam[e];
        Gdf[e] = df_from_double(Gam[e]);
    }
    __syncwarp();
    double md = 0.0;
    for (int i = lane; i < R; i += 32) md = fmax(md, fabs(L[i * ld + i]));
    md = warp_max(md);
    const bool ok = md > 0.0 && warp_cholesky(L, R, ld, 100.0 * rtol * md);
    if (lane == 0) *gam_ok = ok ? 1 : 0;
    if (!ok) return;
    for (int i = lane; i < R; i += 32) rinv[i] = 1.0 / L[i * ld + i];
    __syncwarp();
    // lane c: column c of L⁻¹ by forward substitution (no divisions in the loop)
    for (int c = lane; c < R; c += 32) {
        for (int i = 0; i < R; ++i) {
            double x = 0.0;
            if (i >= c) {
                x = (i == c) ? 1.0 : 0.0;
                for (int q = c; q < i; ++q) x -= L[i * ld + q] * Li[q * ld + c];
                x *= rinv[i];
            }
            Li[i * ld + c] = x;
        }
    }
    __syncwarp();
    for (int e = lane; e < R * R; e += 32) {
        const int i = e / R, q = e % R;
        RV[e] = (q >= i) ? L[q * ld + i] : 0.0;     // R_V = Lᵀ
        Linv[e] = Li[i * ld + q];
        LinvF[e] = (float)Li[i * ld + q];
    }
}

// Q_V = V R_V⁻¹ = V L⁻ᵀ in FP32, one warp per row of V.
static __global__ void k_qv(const double *__restrict__ V, const double *__restrict__ Linv, int J, int R,
                     float *__restrict__ QV) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= J) return;
    for (int c = lane; c < R; c += 32) {
        double s = 0.0;
        for (int t = 0; t <= c; ++t) s += V[(int64_t)j * R + t] * Linv[c * R + t];
        QV[(int64_t)j * R + c] = (float)s;
    }
}

// ---------------------------------------------------------------------------
// Slices the tiles cannot hold (more than FU_TILE_MAX new rows, or several
// segments) are split into chunks of at most FU_TILE_MAX rows of one segment.
//   k_big_b  one warp per chunk: U from P' = X Q_V (computed by k_xv) as in
//            the tiles, written out; chunk partials of ΔD = UᵀU and Δc.
//   k_big_c  one warp per slice (big slices, then untouched slices with no
//            chunks): sums its chunk partials in order, then slice_finish().
// Slices whose S_k has a zero entry take the FP64 map M = S(SΓS)⁺ in k_big_b.
struct BigArgs {
    const float *Y;           // N×R, rows of big slices hold P' = X Q_V
    const int64_t *ch_row0;   // chunk start row
    const int *ch_n;          // chunk rows
    const int *ch_k;          // chunk slice
    int n_chunks;
    const int *fin_k;         // slices to finish: big slices then untouched
    const int *fin_c0;        // [n_fin + 1] chunk range per slice (0 chunks: untouched)
    int n_fin;
    float *dpart;             // n_chunks × (R·R + R)
};

// General Lemma 1 map of slice k (rare: a zero weight or a singular Γ):
// column `lane` of R_V S (S Γ S)⁺ in FP64, rounded into Mo[t][lane].
static __device__ __noinline__ void big_general_map(const FusedArgs &a, int k, float (*Mo)[FU_RP]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = a.R;
    double *wsp = a.wsp + (size_t)(blockIdx.x * FU_WARPS + warp) * fu_wsp_doubles(R);
    const int ld = R + 1;
    double *Aw = wsp, *Ew = Aw + R * ld, *Mw = Ew + R * ld, *fw = Mw + R * ld;
    for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, q = e % R;
        Aw[r * ld + q] = a.W[(int64_t)k * R + r] * a.Gam[e] * a.W[(int64_t)k * R + q];
    }
    __syncwarp();
    warp_psd_pinv(Aw, Ew, fw, Mw, R, ld, a.rtol, 1, false);
    __syncwarp();
    for (int t = 0; t < FU_RP; ++t) {
        double m = 0.0;
        if (t < R && lane < R)
            for (int q = t; q < R; ++q) m += a.RV[t * R + q] * a.W[(int64_t)k * R + q] * Mw[q * ld + lane];
        Mo[t][lane] = (float)m;
    }
    __syncwarp();
    if (lane == 0) atomicAdd(&a.err[1], 1);
}

__device__ __forceinline__ void big_chunk(const FusedArgs &a, const BigArgs &bg, int ch,
                                          float (*Usw)[FU_RP]) {
    const int lane = threadIdx.x & 31;
    const int R = a.R;
    const bool act = lane < R;
    const int k = bg.ch_k[ch];
    const int64_t row0 = bg.ch_row0[ch];
    const int n = bg.ch_n[ch];
    const bool gam_ok = *a.gam_ok != 0;
    const double wold_d = act ? a.W[(int64_t)k * R + lane] : 1.0;
    const bool fast = gam_ok && __all_sync(0xffffffffu, wold_d != 0.0);
    // U = P' mcol: fast path mcol = column `lane` of R_V⁻ᵀ S⁻¹; general path
    // (zero weights) mcol = column of R_V S (S Γ S)⁺ in FP64 (rare), and Δc
    // then needs P' R_V, read from global memory row by row
    float mcol[FU_RP];
    if (fast) {
        const float winv = act ? 1.0f / (float)wold_d : 0.f;
#pragma unroll
        for (int t = 0; t < FU_RP; ++t) mcol[t] = (t < R && act) ? a.GPf[t * R + lane] * winv : 0.f;
    } else {
        big_general_map(a, k, Usw);
#pragma unroll
        for (int t = 0; t < FU_RP; ++t) mcol[t] = Usw[t][lane];
        __syncwarp();
    }
    float dd[FU_RP];
#pragma unroll
    for (int q = 0; q < FU_RP; ++q) dd[q] = 0.f;
    float dc = 0.f;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int m = min(32, n - i0);
        // P' rows → shared (lane = column), loads issued 8 rows at a time
        const float *yb = bg.Y + (row0 + i0) * R + lane;
        for (int i = 0; i < m; i += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = (act && i + u < m) ? yb[(int64_t)(i + u) * R] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i + u < m) Usw[i + u][lane] = v[u];
        }
        __syncwarp();
#pragma unroll 1
        for (int i = 0; i < m; ++i) {
            float u0 = 0.f, u1 = 0.f, u2 = 0.f, u3 = 0.f;
#pragma unroll
            for (int t = 0; t < FU_RP; t += 4) {
                const float4 p4 = *reinterpret_cast<const float4 *>(&Usw[i][t]);
                u0 = fmaf(p4.x, mcol[t], u0);
                u1 = fmaf(p4.y, mcol[t + 1], u1);
                u2 = fmaf(p4.z, mcol[t + 2], u2);
                u3 = fmaf(p4.w, mcol[t + 3], u3);
            }
            const float u = (u0 + u1) + (u2 + u3);
            if (!fast) {
                float pl = 0.f;
                for (int t = 0; t < R; ++t) pl = fmaf(Usw[i][t], act ? (float)a.RV[t * R + lane] : 0.f, pl);
                dc = fmaf(u, pl, dc);
            }
            __syncwarp();
            Usw[i][lane] = u;
            if (act) a.U[(row0 + i0 + i) * R + lane] = u;
        }
        __syncwarp();
#pragma unroll 1
        for (int i = 0; i < m; ++i) {
            const float ul = Usw[i][lane];
#pragma unroll
            for (int q = 0; q < FU_RP; q += 4) {
                const float4 u4 = *reinterpret_cast<const float4 *>(&Usw[i][q]);
                dd[q] = fmaf(ul, u4.x, dd[q]);
                dd[q + 1] = fmaf(ul, u4.y, dd[q + 1]);
                dd[q + 2] = fmaf(ul, u4.z, dd[q + 2]);
                dd[q + 3] = fmaf(ul, u4.w, dd[q + 3]);
            }
        }
        __syncwarp();
    }
    if (fast) {                       // Δc = diag(ΔD S Γ) for this chunk
        // ΔD through shared memory (Usw[q][l] = ΔD[q][l], symmetric), so the
        // loop over q needs no register-indexed dd
#pragma unroll
        for (int q = 0; q < FU_RP; ++q) Usw[q][lane] = dd[q];
        __syncwarp();
        const float wl = act ? (float)wold_d : 0.f;
        float sacc = 0.f;
#pragma unroll 4
        for (int q = 0; q < R; ++q) {
            const float wq = __shfl_sync(0xffffffffu, wl, q);
            if (act) sacc = fmaf(Usw[q][lane] * wq, a.Gdf[q * R + lane].hi, sacc);   // (float)Γ
        }
        __syncwarp();
        dc = sacc;
    }
    // ΔD is symmetric (entry (l, q) and (q, l) are the same FMA sequence), so
    // lane l stores column l: coalesced
    float *out = bg.dpart + (size_t)ch * (R * R + R);
    if (act) {
#pragma unroll
        for (int q = 0; q < FU_RP; ++q)
            if (q < R) out[q * R + lane] = dd[q];
        out[R * R + lane] = dc;
    }
}

static __global__ void __launch_bounds__(256, 2) k_big_b(FusedArgs a, BigArgs bg) {
    __shared__ __align__(16) float Us[FU_WARPS][32][FU_RP];
    const int warp = threadIdx.x >> 5;
    for (int ch = blockIdx.x * FU_WARPS + warp; ch < bg.n_chunks; ch += gridDim.x * FU_WARPS) {
        big_chunk(a, bg, ch, Us[warp]);
    }
}

// chol_solve_reg with L read from the warp's shared block (Lw[l][j], pitch
// FU_LD) in both sweeps: the same operations in the same order, in rolled
// loops (k_big_c keeps its straight-line code short).
__device__ __forceinline__ float chol_solve_smem(const float *Lw, float myinv, bool act, float b) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float y = act ? b : 0.f;
#pragma unroll 4
    for (int j = 0; j < FU_RP; ++j) {
        const float yj = __shfl_sync(full, y * myinv, j);
        if (lane == j) y = yj;
        else if (lane > j) y = fmaf(-Lw[lane * FU_LD + j], yj, y);
    }
#pragma unroll 4
    for (int j = FU_RP - 1; j >= 0; --j) {
        const float xj = __shfl_sync(full, y * myinv, j);
        if (lane == j) y = xj;
        else if (lane < j) y = fmaf(-Lw[j * FU_LD + lane], xj, y);
    }
    return act ? y : 0.f;
}

// FP64 pseudo-inverse solve of W(k,:) (rare: the FP32 factor broke down):
// A = Γ ∗ D_k, b = c_k.  Returns w_k,new[lane].
static __device__ __noinline__ double big_c_fallback(const FusedArgs &a, const df *Dk, df cnew, double *wsp) {
    const int lane = threadIdx.x & 31;
    const int R = a.R;
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
    if (lane == 0) atomicAdd(&a.err[1], 1);
    return lane < R ? bw[lane] : 0.0;
}

#ifndef BC_DB
#define BC_DB 4
#endif
// k_big_c's slice finish: the arithmetic of slice_finish (Eqs. 12, 15-16,
// 21) arranged so that a single R×R block lives in registers across the solve
// and three CTAs fit on an SM.  ΔD is summed from the slice's chunk partials
// once for the D_k update and once more, in the same order (so to the same
// bits), for the slice's share S_k ΔD S_k of G_inc; Γ is read through L1;
// D_k moves as float2 pairs.  gsm is the warp's G block (row `lane`, pitch
// FU_LD).  Called by all 32 lanes of a warp.
__device__ __forceinline__ void big_c_finish(const FusedArgs &a, const BigArgs &bg, int f,
                                             float *Lw, float *gsm, double *wsp) {
    // optional phase clock (profiling, lane 0 adds each phase's cycles):
    // ΔD sums, c/D update, factorisation, triangular solves, refinement
    // residual, W write and G share
    unsigned long long *const pc = a.phase_cycles;
    long long t_ph = pc ? clock64() : 0;
    auto mark = [&](int i) {
        if (pc) {
            const long long t = clock64();
            if ((threadIdx.x & 31) == 0) atomicAdd(pc + i, (unsigned long long)(t - t_ph));
            t_ph = t;
        }
    };
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int R = a.R;
    const bool act = lane < R;
    const int k = bg.fin_k[f];
    const int c0 = bg.fin_c0[f], c1 = bg.fin_c0[f + 1];
    const size_t cst = (size_t)R * R + R;
    const float2 *G2 = reinterpret_cast<const float2 *>(a.Gdf);
    df *Dk = a.D + (int64_t)k * R * R;
    float2 *D2 = reinterpret_cast<float2 *>(Dk);
    const df lamdf{a.lam_hi, a.lam_lo};
    const bool keep_old = a.lam_on != 0;
    // ΔD column `lane` (= row `lane`: ΔD is symmetric) into the warp's shared
    // block Lw, eight rows at a time (each entry summed over the chunks in
    // order), and Δc[lane]; Lw takes the Cholesky factor later
    float dc = 0.f;
    __syncwarp();
#pragma unroll
    for (int q0 = 0; q0 < FU_RP; q0 += 8) {
        float sd[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sd[u] = 0.f;
        if (q0 < R)
            for (int c = c0; c < c1; ++c) {
                const float *in = bg.dpart + (size_t)c * cst;
                if (act) {
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (q0 + u < R) sd[u] += in[(q0 + u) * R + lane];
                    if (q0 == 0) dc += in[R * R + lane];
                }
            }
#pragma unroll
        for (int u = 0; u < 8; ++u) Lw[(q0 + u) * FU_LD + lane] = sd[u];
    }
    __syncwarp();
    mark(0);
    df cnew = {0.f, 0.f};
    if (act) {
        const df cold = a.c[(int64_t)k * R + lane];
        cnew = keep_old ? df_add_f(df_mul(lamdf, cold), dc) : df_make(dc);
        a.c[(int64_t)k * R + lane] = cnew;
    }
    // D_k ← λD_k + ΔD and row `lane` of A = Γ ∗ D_k (hi parts); rows and
    // columns >= R stay zero, so the factorisation runs over all 32 unguarded
    float row[FU_RP];
    float mydiag = 0.f;
#pragma unroll
    for (int r0 = 0; r0 < FU_RP; r0 += BC_DB) {
        float2 dold[BC_DB];
#pragma unroll
        for (int u = 0; u < BC_DB; ++u)
            dold[u] = (r0 + u < R && act && keep_old) ? D2[(r0 + u) * R + lane] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < BC_DB; ++u) {
            const int r = r0 + u;
            row[r] = 0.f;
            if (r < R && act) {
                const float dd = Lw[r * FU_LD + lane];
                const df dn = keep_old ? df_add_f(df_mul(lamdf, df{dold[u].x, dold[u].y}), dd) : df_make(dd);
                D2[r * R + lane] = make_float2(dn.hi, dn.lo);
                const float2 g = __ldg(G2 + r * R + lane);
                // the leading part only, for the FP32 factorisation (the refinement
                // re-forms the product in double-float)
                row[r] = fmaf(g.x, dn.hi, fmaf(g.x, dn.lo, g.y * dn.hi));
                if (r == lane) mydiag = row[r];
            }
        }
    }
    const float amax = warp_max_f(fabsf(mydiag));
    mark(1);
    // right-looking Cholesky of A (hi parts), lane l = row l
    const float tol = 1e-6f * amax;
    bool ok = amax > 0.f;
    float myinv = 0.f;
#pragma unroll 32
    for (int j = 0; j < FU_RP; ++j) {
        const float piv = __shfl_sync(full, row[j], j);
        if (j < R) ok = ok && (piv > tol);
        const float inv = rsqrtf(fmaxf(piv, 1e-30f));
        const float lij = (lane == j) ? piv * inv : row[j] * inv;
        row[j] = lij;
        if (lane == j) myinv = inv;
#pragma unroll 31
        for (int q = j + 1; q < FU_RP; ++q) {
            const float lqj = __shfl_sync(full, lij, q);
            row[q] = fmaf(-lij, lqj, row[q]);
        }
    }
    mark(2);
    df x = {0.f, 0.f};
    if (ok) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < FU_RP; ++j) Lw[lane * FU_LD + j] = row[j];
        __syncwarp();
        const float x0 = chol_solve_smem(Lw, myinv, act, cnew.hi);
        mark(3);
        // one refinement step: res = c − A x0 with A re-formed from the D_k
        // just written (A(lane, r) = ph + pl, ph = Γ.hi·D.hi, pl its error
        // and cross terms).  The sum is carried as s + e, Ogita, Rump and
        // Oishi's Dot2: each ph·x_r and each addition split error-free, the
        // errors and pl·x_r summed in FP32, so s + e is the residual as if
        // formed in twice the working precision.
        float s = cnew.hi, e = cnew.lo;
#pragma unroll 4
        for (int r = 0; r < R; ++r) {
            const float xr = __shfl_sync(full, x0, r);
            if (act) {
                const float2 g = __ldg(G2 + r * R + lane);
                const float2 d = D2[r * R + lane];
                const float ph = g.x * d.x;
                const float pl = fmaf(g.x, d.y, fmaf(g.y, d.x, fmaf(g.x, d.x, -ph)));
                const df q = two_prod(ph, xr);
                const df t = two_sum(s, -q.hi);
                s = t.hi;
                e = fmaf(-pl, xr, __fsub_rn(__fadd_rn(e, t.lo), q.lo));
            }
        }
        mark(4);
        const float dx = chol_solve_smem(Lw, myinv, act, __fadd_rn(s, e));
        x = two_sum(x0, dx);
        ok = __all_sync(full, isfinite(x.hi));
        mark(3);
    }
    double wnew_d;
    if (ok) {
        wnew_d = act ? df_to_double(x) : 0.0;
    } else {
        wnew_d = big_c_fallback(a, Dk, cnew, wsp);
    }
    if (act) a.W[(int64_t)k * R + lane] = wnew_d;
    if (act && a.Wf) a.Wf[(int64_t)k * R + lane] = (float)wnew_d;
    if (act && !isfinite(wnew_d)) atomicAdd(a.err + 2, 1);   // reported as DASH_ENUMERIC
    const float wnew = (float)wnew_d;
    // S_k ΔD S_k, row `lane`, into the warp's G block: ΔD summed again
#pragma unroll 1
    for (int q0 = 0; q0 < R; q0 += 8) {
        float sd[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sd[u] = 0.f;
        for (int c = c0; c < c1; ++c) {
            const float *in = bg.dpart + (size_t)c * cst;
            if (act)
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (q0 + u < R) sd[u] += in[(q0 + u) * R + lane];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u;
            const float wq = __shfl_sync(full, wnew, q);
            if (act && q < R) gsm[lane * FU_LD + q] = fmaf(wnew * sd[u], wq, gsm[lane * FU_LD + q]);
        }
    }
    __syncwarp();
    mark(5);
}

// Three CTAs of eight warps per SM (at most 80 registers a thread); each warp
// finishes whole slices and keeps its G partial in shared memory, the CTA
// sums the eight partials in a fixed order.
static __global__ void __launch_bounds__(256, kBigCBlocksPerSM) k_big_c(FusedArgs a, BigArgs bg, double *Gpart_out) {
    __shared__ __align__(16) float Lw_all[FU_WARPS][FU_RP * FU_LD];
    __shared__ float G_all[FU_WARPS][FU_RP * FU_LD];                  // per-warp G partials
    if (a.err[3]) return;        // a bounded wait of this update timed out: state untouched
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = a.R;
    for (int i = threadIdx.x; i < FU_WARPS * FU_RP * FU_LD; i += blockDim.x) (&G_all[0][0])[i] = 0.f;
    __syncthreads();
    double *wsp = a.wsp + (size_t)(blockIdx.x * FU_WARPS + warp) * fu_wsp_doubles(R);
    // bring the next slice's state (D_k, c_k, W(k,:)) and chunk partials into
    // L2 while this one is finished
    auto prefetch = [&](int f2) {
        if (f2 >= bg.n_fin) return;
        const int k2 = bg.fin_k[f2];
        const char *dk = reinterpret_cast<const char *>(a.D + (int64_t)k2 * R * R);
        for (int l = lane; l < (R * R * 8 + 127) / 128; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(dk + 128 * l));
        if (lane == 0) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(a.c + (int64_t)k2 * R)));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(a.W + (int64_t)k2 * R)));
        }
        const int c0 = bg.fin_c0[f2], c1 = bg.fin_c0[f2 + 1];
        const char *dp = reinterpret_cast<const char *>(bg.dpart + (size_t)c0 * (R * R + R));
        const int nl = (int)(((size_t)(c1 - c0) * (R * R + R) * 4 + 127) / 128);
        for (int l = lane; l < nl; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(dp + 128 * l));
    };
    for (int f = blockIdx.x * FU_WARPS + warp; f < bg.n_fin; f += gridDim.x * FU_WARPS) {
        prefetch(f + gridDim.x * FU_WARPS);
        big_c_finish(a, bg, f, Lw_all[warp], G_all[warp], wsp);
    }
    __syncthreads();
    // the eight warp partials summed in double-float, one conversion to FP64
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int r = e / R, q = e % R;
        df s = df_make(G_all[0][r * FU_LD + q]);
        for (int w = 1; w < FU_WARPS; ++w) s = df_add_f(s, G_all[w][r * FU_LD + q]);
        Gpart_out[(int64_t)blockIdx.x * R * R + e] = df_to_double(s);
    }
}

}  // namespace dash
