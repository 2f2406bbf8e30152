// Streaming tensor-core kernels for the two bulk products of a mode-P update
// when every slice goes through the chunked path (P3 and P5 of Algorithm 1):
//
//   k_xq_tc   P' = X·Q_V for every general row, plus ‖X‖² partials
//             (Theorem 1's X_k,new V term in the V = Q_V R_V basis)
//   k_utilde  Ũ = U ∘ w_k,new per general row (the U_k,new S_k,new of Eq. 20)
//   k_f_tc    per-CTA partials of F_inc = Σ_rows X(i,:)ᵀ Ũ(i,:)  (Eq. 20)
//
// Products: warp-level tensor-core MMAs on the FP16 split x = hi + lo of
// both operands (hi·hi + hi·lo + lo·hi; Ootomo and Yokota 2022).  Operands
// are scaled by powers of two so that their maxima lie in [512, 1024): then a
// lo half that leaves FP16's normal range is below 2^-35 of the maximum, and
// each operand keeps ~22 significant bits.  Every k-step (or group of
// k-steps with one scale) starts a fresh MMA accumulator, which is scaled
// back and added to the FP32 running sum with a rounded FMA.
//
// Data movement: each thread copies exactly the float4s it will later read
// into its own shared-memory slots with cp.async, several stages ahead, and
// waits only on its own copy groups (cp.async.wait_group): deep memory-level
// parallelism without register cost and without any cross-thread wait.
//
// A sum over a contraction index does not depend on the order of its terms,
// so each kernel assigns the MMA's k (and m/n) slots to columns or rows in
// whatever order makes a thread's values contiguous in memory, and applies
// the same assignment to the other operand.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dash_kernels_fused.cuh"
#include "dash_kernels_p.cuh"

namespace dash {

constexpr int XQ_THREADS = 256;
constexpr int XQ_WARPS = XQ_THREADS / 32;
constexpr int XQ_KU = 4;                  // k-steps per stage (one scale per row)
constexpr int XQ_S = 4;                   // stages in flight per warp

__device__ __forceinline__ uint32_t xq_h2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
// FP16 (hi, lo) halves of a pair already scaled into range
__device__ __forceinline__ void xq_split(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = xq_h2(x0 - hf.x, x1 - hf.y);
}
__device__ __forceinline__ void xq_mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                       uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// 2^e as a float, for -126 <= e <= 127
__device__ __forceinline__ float xq_pow2(int e) { return __int_as_float((127 + e) << 23); }
// e with m = f·2^e, f in [0.5, 1), for finite m >= 0, clamped below at -60 (a
// zero or tiny maximum gives a bounded scale: values all below 2^-60 are
// scaled by at most 2^70)
__device__ __forceinline__ int xq_exp(float m) {
    const int e = ((__float_as_int(m) >> 23) & 0xff) - 126;
    return e < -60 ? -60 : e;
}
__device__ __forceinline__ float fmax4(float4 v) {
    return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
}
__device__ __forceinline__ float4 f4scale(float4 v, float s) {
    return make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
}

// per-thread asynchronous copies global → shared; `valid` false fills zeros
// (source size 0, nothing read)
__device__ __forceinline__ void cpa16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Power-of-two exponent bexp that brings max |B| into [512, 1024), clamped
// to [-40, 40]; B is J×R.  One warp.
static __global__ void k_xq_bscale(const float *__restrict__ B, int n, int *__restrict__ bexp) {
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += 32) m = fmaxf(m, fabsf(B[i]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
        int e = 10 - (((__float_as_int(m) >> 23) & 0xff) - 126);
        if (m == 0.f) e = 0;
        *bexp = e < -40 ? -40 : (e > 40 ? 40 : e);
    }
}

// B fragments for k_xq_tc: B (J×R FP32, row-major) times 2^bexp, split.
// Fragment (ks, nt), lane (g = lane/4, tg = lane%4), holds {b0hi, b1hi, b0lo,
// b1lo}: k-slots 2tg, 2tg+1 (b0) and 2tg+8, 2tg+9 (b1) are columns j =
// 16ks + 4tg + {0, 1} and {2, 3}; n-slot g is rank column 8nt + g.  Entries
// past J or R are 0.
static __global__ void k_xq_bfrag(const float *__restrict__ B, int J, int R,
                                  const int *__restrict__ bexp, uint4 *__restrict__ frag) {
    const int nks = (J + 15) / 16, nnt = (R + 7) / 8;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nks * nnt * 32) return;
    const int lane = i % 32, nt = (i / 32) % nnt, ks = i / (32 * nnt);
    const int g = lane >> 2, tg = lane & 3;
    const int n = 8 * nt + g;
    const float sc = xq_pow2(*bexp);
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = 16 * ks + 4 * tg + q;
        v[q] = (j < J && n < R) ? B[(int64_t)j * R + n] * sc : 0.f;
    }
    uint4 f;
    xq_split(v[0], v[1], f.x, f.z);
    xq_split(v[2], v[3], f.y, f.w);
    frag[i] = f;
}

// Row g of the general rows: one run (the split plan: every row of the batch,
// in order) maps with an add, otherwise gen_row's search.
__device__ __forceinline__ int64_t run0_of(const BatchDev &b) {
    return b.n_runs == 1 ? b.run_row0[0] : -1;
}
__device__ __forceinline__ int64_t gen_row_fast(const BatchDev &b, int64_t run0, int64_t g) {
    return run0 >= 0 ? run0 + g : gen_row(b, g);
}

// Dynamic shared memory of k_xq_tc: the B fragments, then per warp XQ_S
// stages of XQ_KU k-steps × 2 rows of float4 per lane.
__host__ __device__ inline size_t xq_smem(int J, int R) {
    return (size_t)((J + 15) / 16) * ((R + 7) / 8) * 32 * 16 +
           (size_t)XQ_WARPS * XQ_S * XQ_KU * 2 * 32 * 16;
}

// P(row, :) = X(row, :)·B for the N_gen general rows (general row g lives at
// gen_row(b, g)); per-CTA partial of Σ ‖x‖² in xn_part[blockIdx.x]; xe[g] =
// the exponent e of the row's max |x| (max = f·2^e, f in [0.5, 1)).  A warp
// takes 16-row tiles.  Lane (g = lane/4, tg = lane%4) holds rows g and g+8
// of the tile; in k-step kk its k-slots 2tg, 2tg+1, 2tg+8, 2tg+9 are columns
// 16kk + 4tg + {0, 1, 2, 3} (one float4 per row).  A stage is XQ_KU k-steps;
// each row is scaled once per stage (max over its 64 columns).
// Requires J % 4 == 0, 16-byte aligned rows and R <= 32.
static __global__ void __launch_bounds__(XQ_THREADS, 1)
    k_xq_tc(const float *__restrict__ X, BatchDev b, int J, int R, const uint4 *__restrict__ frag,
            const int *__restrict__ bexp_p, float *__restrict__ P, double *__restrict__ xn_part,
            int *__restrict__ xe) {
    extern __shared__ uint4 xq_sm[];
    const int nks = (J + 15) / 16, nnt = (R + 7) / 8;
    const int nfr = nks * nnt * 32;
    for (int i = threadIdx.x; i < nfr; i += XQ_THREADS) xq_sm[i] = frag[i];
    __syncthreads();
    const float bunscale = xq_pow2(-*bexp_p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    float4 *ring = reinterpret_cast<float4 *>(xq_sm + nfr) + (size_t)warp * XQ_S * XQ_KU * 2 * 32 + lane;
    const int64_t run0 = run0_of(b);
    const int64_t Ng = b.N_gen;
    const int64_t ntile = (Ng + 15) / 16;
    const int64_t t0 = (int64_t)blockIdx.x * XQ_WARPS + warp, tstride = (int64_t)gridDim.x * XQ_WARPS;
    const int nkg = (nks + XQ_KU - 1) / XQ_KU;
    const int ntw = t0 < ntile ? (int)((ntile - 1 - t0) / tstride + 1) : 0;
    const int total = ntw * nkg;
    // stage cursor of the copies (runs XQ_S - 1 stages ahead): tile, k-group
    int is = 0, itile = 0, ikg = 0;
    const float *xa = X, *xb = X;
    bool iva = false, ivb = false;
    auto issue = [&]() {
        if (is < total) {
            if (ikg == 0) {
                const int64_t ga = 16 * (t0 + (int64_t)itile * tstride) + g, gb = ga + 8;
                iva = ga < Ng;
                ivb = gb < Ng;
                xa = X + (iva ? gen_row_fast(b, run0, ga) : 0) * (int64_t)J + 4 * tg;
                xb = X + (ivb ? gen_row_fast(b, run0, gb) : 0) * (int64_t)J + 4 * tg;
            }
            float4 *slot = ring + (is & (XQ_S - 1)) * XQ_KU * 2 * 32;
#pragma unroll
            for (int u = 0; u < XQ_KU; ++u) {
                const int kk = ikg * XQ_KU + u;
                const int j0 = 16 * kk;
                const bool c = kk < nks && j0 + 4 * tg < J;
                cpa16(slot + (2 * u) * 32, (iva && c) ? xa + j0 : X, iva && c);
                cpa16(slot + (2 * u + 1) * 32, (ivb && c) ? xb + j0 : X, ivb && c);
            }
            if (++ikg == nkg) {
                ikg = 0;
                ++itile;
            }
        }
        ++is;
        cpa_commit();
    };
#pragma unroll
    for (int i = 0; i < XQ_S - 1; ++i) issue();
    double xn = 0.0;
    float xnf = 0.f, rm0 = 0.f, rm1 = 0.f;
    float acc[4][4];
    int ctile = 0, kg = 0;
    for (int i = 0; i < total; ++i) {
        issue();
        cpa_wait<XQ_S - 1>();
        if (kg == 0) {
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
            xnf = 0.f;
            rm0 = rm1 = 0.f;
        }
        const float4 *slot = ring + (i & (XQ_S - 1)) * XQ_KU * 2 * 32;
        float4 xv[XQ_KU][2];
        float m0 = 0.f, m1 = 0.f;
#pragma unroll
        for (int u = 0; u < XQ_KU; ++u) {
            xv[u][0] = slot[(2 * u) * 32];
            xv[u][1] = slot[(2 * u + 1) * 32];
            const float4 p = xv[u][0], q = xv[u][1];
            xnf += p.x * p.x + p.y * p.y + p.z * p.z + p.w * p.w +
                   q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
            m0 = fmaxf(m0, fmax4(p));
            m1 = fmaxf(m1, fmax4(q));
        }
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
        rm0 = fmaxf(rm0, m0);
        rm1 = fmaxf(rm1, m1);
        const int e0 = xq_exp(m0), e1 = xq_exp(m1);
        const float s0 = xq_pow2(10 - e0), s1 = xq_pow2(10 - e1);
        float d[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[nt][e] = 0.f;
#pragma unroll
        for (int u = 0; u < XQ_KU; ++u) {
            const int kk = kg * XQ_KU + u;
            if (kk < nks) {
                const float4 p = f4scale(xv[u][0], s0), q = f4scale(xv[u][1], s1);
                uint32_t a0h, a0l, a1h, a1l, a2h, a2l, a3h, a3l;
                xq_split(p.x, p.y, a0h, a0l);      // row g,   k 2tg, 2tg+1
                xq_split(q.x, q.y, a1h, a1l);      // row g+8
                xq_split(p.z, p.w, a2h, a2l);      // row g,   k 2tg+8, 2tg+9
                xq_split(q.z, q.w, a3h, a3l);      // row g+8
                const uint4 *fr = xq_sm + (size_t)kk * nnt * 32 + lane;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    if (nt < nnt) {
                        const uint4 f = fr[nt * 32];
                        xq_mma(d[nt], a0h, a1h, a2h, a3h, f.x, f.y);
                        xq_mma(d[nt], a0h, a1h, a2h, a3h, f.z, f.w);
                        xq_mma(d[nt], a0l, a1l, a2l, a3l, f.x, f.y);
                    }
                }
            }
        }
        const float u0 = xq_pow2(e0 - 10), u1 = xq_pow2(e1 - 10);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            acc[nt][0] = fmaf(d[nt][0], u0, acc[nt][0]);
            acc[nt][1] = fmaf(d[nt][1], u0, acc[nt][1]);
            acc[nt][2] = fmaf(d[nt][2], u1, acc[nt][2]);
            acc[nt][3] = fmaf(d[nt][3], u1, acc[nt][3]);
        }
        if (++kg == nkg) {
            kg = 0;
            xn += (double)xnf;
            const int64_t ga = 16 * (t0 + (int64_t)ctile * tstride) + g, gb = ga + 8;
            ++ctile;
            const bool va = ga < Ng, vb = gb < Ng;
            const int64_t ra = va ? gen_row_fast(b, run0, ga) : 0, rb = vb ? gen_row_fast(b, run0, gb) : 0;
            if (tg == 0) {
                if (va) xe[ga] = xq_exp(rm0);
                if (vb) xe[gb] = xq_exp(rm1);
            }
            // rows ga (acc[.][0..1]) and gb (acc[.][2..3]), columns 8nt + 2tg, +1
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = 8 * nt + 2 * tg;
                if (va && c < R) P[ra * R + c] = acc[nt][0] * bunscale;
                if (va && c + 1 < R) P[ra * R + c + 1] = acc[nt][1] * bunscale;
                if (vb && c < R) P[rb * R + c] = acc[nt][2] * bunscale;
                if (vb && c + 1 < R) P[rb * R + c + 1] = acc[nt][3] * bunscale;
            }
        }
    }
    cpa_wait<0>();
    xn = warp_sum(xn);
    __shared__ double red[XQ_WARPS];
    if (lane == 0) red[warp] = xn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < XQ_WARPS; ++w) s += red[w];
        xn_part[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Ũ for k_f_tc, one CTA of 128 threads per 16-row group G of the general
// rows: Ũ(g, :) = U(row, :) ∘ w_k,new (rounded once from the FP64 product),
// scaled by 2^(10 - eu) with eu the exponent of the group's max |Ũ|, in FP32
// with row pitch `pitch` (8·⌈R/8⌉; columns R.. zero); gex[G] = {ex, eu} with
// ex the largest row exponent xe of the group's rows (the X scale k_f_tc
// applies to all 16 rows).  Thread t: row 16G + t/8, columns 4(t%8) ...
static __global__ void __launch_bounds__(128) k_utilde(BatchDev b, int R, int pitch,
                                                       const float *__restrict__ U,
                                                       const double *__restrict__ W,
                                                       const int *__restrict__ xe,
                                                       float *__restrict__ Ut, int2 *__restrict__ gex) {
    __shared__ float smx[4];
    __shared__ int sex[4];
    const int t = threadIdx.x, q = t & 7;
    const int64_t gg = 16 * (int64_t)blockIdx.x + (t >> 3);
    const bool rowok = gg < b.N_gen;
    const bool ok = rowok && 4 * q < pitch;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    int ex = -60;
    if (rowok) ex = xe[gg];
    if (ok) {
        const int64_t row = gen_row_fast(b, run0_of(b), gg);
        const int k = b.row_slice[row];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int r = 4 * q + c;
            v[c] = r < R ? (float)((double)U[row * R + r] * W[(int64_t)k * R + r]) : 0.f;
        }
    }
    float m = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    }
    if ((t & 31) == 0) {
        smx[t >> 5] = m;
        sex[t >> 5] = ex;
    }
    __syncthreads();
    const float mx = fmaxf(fmaxf(smx[0], smx[1]), fmaxf(smx[2], smx[3]));
    const int exg = max(max(sex[0], sex[1]), max(sex[2], sex[3]));
    const int eu = xq_exp(mx);
    const float ts = xq_pow2(10 - eu);
    if (ok)
        reinterpret_cast<float4 *>(Ut + gg * pitch)[q] =
            make_float4(v[0] * ts, v[1] * ts, v[2] * ts, v[3] * ts);
    if (t == 0) gex[blockIdx.x] = make_int2(exg, eu);
}

// ---------------------------------------------------------------------------
// k_f_tc: F partials.  CTA (bx, by) takes the general rows
// [bx·rows_per_cta, ...) (rows_per_cta a multiple of 16, so its k-steps are
// k_utilde's groups) and the columns [512·by, 512·by + 512).  Warp w takes
// column group jg = w % njg (64 columns) and the k-steps (16 rows)
// ks ≡ w / njg (mod nrs) of the CTA's rows, njg = column groups of this CTA,
// nrs = FT_WARPS / njg.
//
// MMA orientation: D (16 j × 8 r) += Xᵀ (16 j × 16 rows) · Ũ (16 rows × 8 r).
// Lane (g, tg) holds the k-slots (rows) 2tg, 2tg+1, 2tg+8, 2tg+9 of the
// k-step; for m-tile t its m-slots g and g+8 are columns
// jg0 + 32(t/2) + 4g + 2(t%2) + {0, 1}, so the lane reads each row as two
// float4s (columns jg0 + 4g and jg0 + 32 + 4g); n-slot g of n-tile nt is
// rank column NT·g + nt, so the lane reads Ũ(row, NT·g .. NT·g + NT - 1).
// The k-step's X is scaled by 2^(10 - ex), its Ũ comes scaled by 2^(10 - eu)
// ({ex, eu} from k_utilde), and its product is scaled back by 2^(ex + eu - 20).
constexpr int FT_THREADS = 256;
constexpr int FT_WARPS = FT_THREADS / 32;
constexpr int FT_S = 4;                   // k-steps in flight per warp (a power of 2)
constexpr int FT_JCTA = 512;              // columns per CTA (8 groups of 64)
constexpr int FT_SLOT = 13;               // float4 per lane per stage: 8 of X, 4 of Ũ, 1 scale

__host__ __device__ inline size_t ft_smem() { return (size_t)FT_WARPS * FT_S * FT_SLOT * 32 * 16; }

template <int NT>
__global__ void __launch_bounds__(FT_THREADS, 1)
    k_f_tc(const float *__restrict__ X, BatchDev b, int J, int R, const float *__restrict__ Ut,
           const int2 *__restrict__ gex, int64_t rows_per_cta, float *__restrict__ Fpart) {
    extern __shared__ float4 ft_sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int jc0 = FT_JCTA * blockIdx.y;
    const int jcn = min(FT_JCTA, J - jc0);
    const int njg = (jcn + 63) / 64;
    const int nrs = FT_WARPS / njg;
    const int jg = warp % njg, rs = warp / njg;
    const bool active = rs < nrs;
    const int jg0 = jc0 + 64 * jg;
    const bool c0ok = jg0 + 4 * g < J, c1ok = jg0 + 32 + 4 * g < J;
    const int64_t run0 = run0_of(b);
    const int64_t gbeg = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t gend = b.N_gen < gbeg + rows_per_cta ? b.N_gen : gbeg + rows_per_cta;
    const int nks = (int)((gend - gbeg + 15) / 16);
    const int my_n = (active && rs < nks) ? (nks - 1 - rs) / nrs + 1 : 0;
    float4 *ring = ft_sm + (size_t)warp * FT_S * FT_SLOT * 32 + lane;
    const int roff[4] = {2 * tg, 2 * tg + 1, 2 * tg + 8, 2 * tg + 9};
    int is = 0;
    int64_t ig0 = gbeg + 16 * rs;             // first row of the next k-step to copy
    auto issue = [&]() {
        if (is < my_n) {
            float4 *slot = ring + (is & (FT_S - 1)) * FT_SLOT * 32;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int64_t gr = ig0 + roff[p];
                const bool rv = gr < gend;
                const float *xr = X + (rv ? gen_row_fast(b, run0, gr) : 0) * (int64_t)J + jg0 + 4 * g;
                cpa16(slot + (2 * p) * 32, (rv && c0ok) ? xr : X, rv && c0ok);
                cpa16(slot + (2 * p + 1) * 32, (rv && c1ok) ? xr + 32 : X, rv && c1ok);
                const float *ur = rv ? Ut + gr * (8 * NT) + NT * g : Ut;
                float *ud = reinterpret_cast<float *>(slot + (8 + p) * 32);
                if constexpr (NT == 4) {
                    cpa16(ud, ur, rv);
                } else if constexpr (NT == 2) {
                    cpa8(ud, ur, rv);
                } else {
#pragma unroll
                    for (int c = 0; c < NT; ++c) cpa4(ud + c, rv ? ur + c : Ut, rv);
                }
            }
            cpa8(slot + 12 * 32, gex + ig0 / 16, true);
            ig0 += 16 * nrs;
        }
        ++is;
        cpa_commit();
    };
#pragma unroll
    for (int i = 0; i < FT_S - 1; ++i) issue();
    float acc[4][NT][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[t][nt][e] = 0.f;
    for (int i = 0; i < my_n; ++i) {
        issue();
        cpa_wait<FT_S - 1>();
        const float4 *slot = ring + (i & (FT_S - 1)) * FT_SLOT * 32;
        const int2 sc = *reinterpret_cast<const int2 *>(slot + 12 * 32);
        const float sx = xq_pow2(10 - sc.x), tu = xq_pow2(sc.x - 10) * xq_pow2(sc.y - 10);
        float4 xv[4][2];
        float4 uv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            xv[p][0] = f4scale(slot[(2 * p) * 32], sx);
            xv[p][1] = f4scale(slot[(2 * p + 1) * 32], sx);
            uv[p] = slot[(8 + p) * 32];
        }
        uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const float u0 = nt == 0 ? uv[0].x : nt == 1 ? uv[0].y : nt == 2 ? uv[0].z : uv[0].w;
            const float u1 = nt == 0 ? uv[1].x : nt == 1 ? uv[1].y : nt == 2 ? uv[1].z : uv[1].w;
            const float u2 = nt == 0 ? uv[2].x : nt == 1 ? uv[2].y : nt == 2 ? uv[2].z : uv[2].w;
            const float u3 = nt == 0 ? uv[3].x : nt == 1 ? uv[3].y : nt == 2 ? uv[3].z : uv[3].w;
            xq_split(u0, u1, bh[nt][0], bl[nt][0]);
            xq_split(u2, u3, bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int q = t >> 1;
            float v[4][2];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float4 x4 = xv[p][q];
                v[p][0] = (t & 1) ? x4.z : x4.x;
                v[p][1] = (t & 1) ? x4.w : x4.y;
            }
            uint32_t a0h, a0l, a1h, a1l, a2h, a2l, a3h, a3l;
            xq_split(v[0][0], v[1][0], a0h, a0l);     // m g,   k 2tg, 2tg+1
            xq_split(v[0][1], v[1][1], a1h, a1l);     // m g+8
            xq_split(v[2][0], v[3][0], a2h, a2l);     // m g,   k 2tg+8, 2tg+9
            xq_split(v[2][1], v[3][1], a3h, a3l);     // m g+8
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                xq_mma(d, a0h, a1h, a2h, a3h, bh[nt][0], bh[nt][1]);
                xq_mma(d, a0h, a1h, a2h, a3h, bl[nt][0], bl[nt][1]);
                xq_mma(d, a0l, a1l, a2l, a3l, bh[nt][0], bh[nt][1]);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[t][nt][e] = fmaf(d[e], tu, acc[t][nt][e]);
            }
        }
    }
    cpa_wait<0>();
    // warps of one column group (row subgroups 1.., in order) add into row
    // subgroup 0, which writes the CTA's partial; the rings are free now
    float *red_all = reinterpret_cast<float *>(ft_sm);
    for (int rr = 1; rr < nrs; ++rr) {
        __syncthreads();
        float *red = red_all + jg * 512 * NT;
        if (active && rs == rr) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) red[((t * NT + nt) * 4 + e) * 32 + lane] = acc[t][nt][e];
        }
        __syncthreads();
        if (active && rs == 0) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[t][nt][e] += red[((t * NT + nt) * 4 + e) * 32 + lane];
        }
    }
    if (active && rs == 0) {
        float *out = Fpart + (int64_t)blockIdx.x * J * R;
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = jg0 + 32 * (t >> 1) + 4 * g + 2 * (t & 1) + (e >> 1);
                    const int r = NT * (2 * tg + (e & 1)) + nt;
                    if (j < J && r < R) out[(int64_t)j * R + r] = acc[t][nt][e];
                }
    }
}

}  // namespace dash
