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
// k-steps with one scale) starts fresh MMA accumulators, one for the hi·hi
// terms and one for the two correction terms, which are scaled back and added
// to the FP32 running sum with rounded FP32 arithmetic.
//
// Data movement: each warp streams its own stages of X (16 rows × 64
// columns) through a ring in shared memory with 1-D bulk copies (one copy per
// row segment, issued by up to 32 lanes at once), each stage completing on
// its own mbarrier.  The warp is both producer and consumer of its ring, so
// no wait depends on another warp; every wait is bounded.  Rows are padded
// in shared memory so that the fragment reads are free of bank conflicts.
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
// d = a·b (fresh accumulator: C is the constant 0)
__device__ __forceinline__ void xq_mma0(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.f));
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

// Bounded wait of a whole warp on its own stage barrier: false after ~1 s
// (counted once in err[0]; err[3] marks the update as abandoned).
__device__ __forceinline__ bool sb_wait(uint64_t *bar, uint32_t parity, int *err) {
    bool got = true;
    if (!mbar_try_wait(bar, parity)) {
        const long long t0 = clock64();
        while (!mbar_try_wait(bar, parity)) {
            if (clock64() - t0 > 2000000000LL) {
                got = false;
                break;
            }
        }
    }
    got = __all_sync(0xffffffffu, got);
    if (!got && (threadIdx.x & 31) == 0) {
        atomicAdd(err, 1);
        err[3] = 1;
    }
    return got;
}

// Row g of the general rows: one run (the split plan: every row of the batch,
// in order) maps with an add, otherwise gen_row's search.
__device__ __forceinline__ int64_t run0_of(const BatchDev &b) {
    return b.n_runs == 1 ? b.run_row0[0] : -1;
}
__device__ __forceinline__ int64_t gen_row_fast(const BatchDev &b, int64_t run0, int64_t g) {
    return run0 >= 0 ? run0 + g : gen_row(b, g);
}

// X scale exponent from a row (or row group) max |x| = f·2^ex, f in [0.5, 1):
// the scale 2^(10 - ex) brings that max into [512, 1024).
__host__ __device__ inline int ft_xscale_exp(int ex) { return 10 - ex; }

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

// ---------------------------------------------------------------------------
// k_xq_tc.  A warp takes 16-row tiles of the general rows; a stage is the
// tile's next 64 columns (4 k-steps, one scale per row).  Lane (g = lane/4,
// tg = lane%4) holds rows g and g+8; in k-step kk its k-slots 2tg, 2tg+1,
// 2tg+8, 2tg+9 are columns 16kk + 4tg + {0, 1, 2, 3} (one float4 per row).
constexpr int XQ_THREADS = 512;
constexpr int XQ_WARPS = XQ_THREADS / 32;
constexpr int XQ_KU = 4;                  // k-steps per stage
constexpr int XQ_S = 2;                   // stages per warp ring (a power of 2)
constexpr int XQ_XP = 80;                 // floats per staged row (≡ 16 mod 32: conflict-free)
constexpr int XQ_STAGE = 16 * XQ_XP;      // floats per stage

// Dynamic shared memory of k_xq_tc: the B fragments, the warps' rings, their
// stage barriers.
__host__ __device__ inline size_t xq_smem(int J, int R) {
    return (size_t)((J + 15) / 16) * ((R + 7) / 8) * 32 * 16 +
           (size_t)XQ_WARPS * XQ_S * XQ_STAGE * 4 + (size_t)XQ_WARPS * XQ_S * 8;
}

// P(row, :) = X(row, :)·B for the N_gen general rows (general row g lives at
// gen_row(b, g)); per-CTA partial of Σ ‖x‖² in xn_part[blockIdx.x]; xe[g] =
// the exponent e of the row's max |x| (max = f·2^e, f in [0.5, 1)).
// Requires J % 4 == 0, 16-byte aligned rows and R <= 32.
static __global__ void __launch_bounds__(XQ_THREADS, 1)
    k_xq_tc(const float *__restrict__ X, BatchDev b, int J, int R, const uint4 *__restrict__ frag,
            const int *__restrict__ bexp_p, float *__restrict__ P, double *__restrict__ xn_part,
            int *__restrict__ xe, int *__restrict__ err, unsigned long long *__restrict__ pc) {
    extern __shared__ __align__(16) uint4 xq_sm[];
    const int nks = (J + 15) / 16, nnt = (R + 7) / 8;
    const int nfr = nks * nnt * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    float *ring = reinterpret_cast<float *>(xq_sm + nfr) + (size_t)warp * XQ_S * XQ_STAGE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<float *>(xq_sm + nfr) +
                                                  (size_t)XQ_WARPS * XQ_S * XQ_STAGE) + warp * XQ_S;
    for (int i = threadIdx.x; i < nfr; i += XQ_THREADS) xq_sm[i] = frag[i];
    if (lane == 0) {
        for (int s = 0; s < XQ_S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const float bunscale = xq_pow2(-*bexp_p);
    const int64_t run0 = run0_of(b);
    const int64_t Ng = b.N_gen;
    const int64_t ntile = (Ng + 15) / 16;
    const int64_t t0 = (int64_t)blockIdx.x * XQ_WARPS + warp, tstride = (int64_t)gridDim.x * XQ_WARPS;
    const int nkg = (J + 63) / 64;
    const int ntw = t0 < ntile ? (int)((ntile - 1 - t0) / tstride + 1) : 0;
    const int total = ntw * nkg;
    // copy cursor (runs XQ_S - 1 stages ahead of the compute): stage, tile, k-group
    int is = 0, itile = 0, ikg = 0;
    const float *isrc = X;                 // this lane's row (lanes 0..15) of the copy tile
    int inv = 0;                           // valid rows of the copy tile
    auto issue = [&]() {
        if (is >= total) return;
        if (ikg == 0) {
            const int64_t r0 = 16 * (t0 + (int64_t)itile * tstride);
            inv = (int)(Ng - r0 < 16 ? Ng - r0 : 16);
            isrc = X + (lane < inv ? gen_row_fast(b, run0, r0 + lane) : 0) * (int64_t)J;
        }
        const int s = is & (XQ_S - 1);
        const uint32_t rb = (uint32_t)min(64, J - 64 * ikg) * 4;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane == 0) mbar_expect_tx(&bars[s], rb * (uint32_t)inv);
        __syncwarp();
        if (lane < inv) bulk_g2s(ring + (size_t)s * XQ_STAGE + lane * XQ_XP, isrc + 64 * ikg, rb, &bars[s]);
        if (++ikg == nkg) {
            ikg = 0;
            ++itile;
        }
        ++is;
    };
#pragma unroll
    for (int i = 0; i < XQ_S - 1; ++i) issue();
    double xn = 0.0;
    float xnf = 0.f, rm0 = 0.f, rm1 = 0.f;
    float acc[4][4];
    int ctile = 0, kg = 0;
    bool aborted = false;
    int i = 0;
    long long cw = 0;                      // profiling: cycles waiting on stages
    const long long c0 = pc ? clock64() : 0;
    for (; i < total; ++i) {
        issue();
        const int s = i & (XQ_S - 1);
        const long long w0 = pc ? clock64() : 0;
        if (!sb_wait(&bars[s], (uint32_t)(i / XQ_S) & 1u, err)) {
            aborted = true;
            break;
        }
        if (pc) cw += clock64() - w0;
        if (kg == 0) {
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
            xnf = 0.f;
            rm0 = rm1 = 0.f;
        }
        const int64_t ga = 16 * (t0 + (int64_t)ctile * tstride) + g, gb = ga + 8;
        const bool va = ga < Ng, vb = gb < Ng;
        const float *st = ring + (size_t)s * XQ_STAGE;
        float4 xv[XQ_KU][2];
        float m0 = 0.f, m1 = 0.f;
#pragma unroll
        for (int u = 0; u < XQ_KU; ++u) {
            const int col = 64 * kg + 16 * u + 4 * tg;
            const bool c = col < J;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            xv[u][0] = (va && c) ? *reinterpret_cast<const float4 *>(st + g * XQ_XP + 16 * u + 4 * tg) : z;
            xv[u][1] = (vb && c) ? *reinterpret_cast<const float4 *>(st + (g + 8) * XQ_XP + 16 * u + 4 * tg) : z;
            const float4 p = xv[u][0], q = xv[u][1];
            xnf += p.x * p.x + p.y * p.y + p.z * p.z + p.w * p.w +
                   q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
            m0 = fmaxf(m0, fmax4(p));
            m1 = fmaxf(m1, fmax4(q));
        }
        __syncwarp();                      // stage s is read: free for its next copy
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
        m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
        rm0 = fmaxf(rm0, m0);
        rm1 = fmaxf(rm1, m1);
        const int x0 = ft_xscale_exp(xq_exp(m0)), x1 = ft_xscale_exp(xq_exp(m1));
        {
            const float s0 = xq_pow2(x0), s1 = xq_pow2(x1);
#pragma unroll
            for (int u = 0; u < XQ_KU; ++u) {
                xv[u][0] = f4scale(xv[u][0], s0);
                xv[u][1] = f4scale(xv[u][1], s1);
            }
        }
        // main (hi·hi) and correction (hi·lo + lo·hi) terms in separate MMA
        // accumulators, added in FP32 after the stage: the small corrections
        // never pass through the accumulator that holds the large terms
        float d[4][4], dc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[nt][e] = dc[nt][e] = 0.f;
#pragma unroll
        for (int u = 0; u < XQ_KU; ++u) {
            const int kk = kg * XQ_KU + u;
            if (kk < nks) {
                const float4 p = xv[u][0], q = xv[u][1];
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
                        xq_mma(dc[nt], a0h, a1h, a2h, a3h, f.z, f.w);
                        xq_mma(dc[nt], a0l, a1l, a2l, a3l, f.x, f.y);
                    }
                }
            }
        }
        const float u0 = xq_pow2(-x0), u1 = xq_pow2(-x1);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            acc[nt][0] = fmaf(d[nt][0] + dc[nt][0], u0, acc[nt][0]);
            acc[nt][1] = fmaf(d[nt][1] + dc[nt][1], u0, acc[nt][1]);
            acc[nt][2] = fmaf(d[nt][2] + dc[nt][2], u1, acc[nt][2]);
            acc[nt][3] = fmaf(d[nt][3] + dc[nt][3], u1, acc[nt][3]);
        }
        if (++kg == nkg) {
            kg = 0;
            ++ctile;
            xn += (double)xnf;
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
    if (aborted) {                         // let the copies already issued land
        for (int k = i; k < is; ++k) sb_wait(&bars[k & (XQ_S - 1)], (uint32_t)(k / XQ_S) & 1u, err);
    }
    if (pc && lane == 0) {
        atomicAdd(&pc[0], (unsigned long long)cw);
        atomicAdd(&pc[1], (unsigned long long)(clock64() - c0));
    }
    xn = warp_sum(xn);
    __shared__ double red[XQ_WARPS];
    if (lane == 0) red[warp] = xn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < XQ_WARPS; ++w) sum += red[w];
        xn_part[blockIdx.x] = sum;
    }
}

// ---------------------------------------------------------------------------
// Ũ for k_f_tc as MMA B fragments, one warp per 16-row group G of the
// general rows.  Ũ(g, r) = U(row, r)·w_k,new(r) (FP32 product with the FP32
// copy of w_new: the FP64 pipe is far too narrow for a per-row product) is
// scaled by 2^(10 - eu), eu the exponent of the group's max |Ũ|,
// and split into FP16 hi + lo.  Block G (ft_ublk(NT) 32-bit words at
// Uf + G·ft_ublk(NT)) holds, for n-tile nt and lane L = (g, tg), the word
// quadruple {bh0, bh1, bl0, bl1} at words 4(32nt + L) ..: bh0 packs the hi
// halves of Ũ(16G + 2tg, NT·g + nt) and Ũ(16G + 2tg + 1, ·), bh1 those of
// rows 2tg + 8 and 2tg + 9, bl0/bl1 the lo halves; then the record
// {sxe, eu, 0, 0}, sxe the X scale exponent of the group (ft_xscale_exp of
// its largest row exponent xe).  Rows past N_gen and columns past R are 0.
__host__ __device__ constexpr int ft_ublk(int NT) { return 128 * NT + 4; }

template <int NT>
__global__ void __launch_bounds__(256) k_utilde(BatchDev b, int R, const float *__restrict__ U,
                                                const float *__restrict__ Wf,
                                                const int *__restrict__ xe,
                                                uint32_t *__restrict__ Uf) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    const int64_t G = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (16 * G >= b.N_gen) return;
    const int64_t run0 = run0_of(b);
    const int roff[4] = {2 * tg, 2 * tg + 1, 2 * tg + 8, 2 * tg + 9};
    float v[4][NT];
    float m = 0.f;
    int ex = -60;
    if (lane < 16 && 16 * G + lane < b.N_gen) ex = __ldcg(xe + 16 * G + lane);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t gg = 16 * G + roff[p];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) v[p][nt] = 0.f;
        if (gg < b.N_gen) {
            const int64_t row = gen_row_fast(b, run0, gg);
            const int k = __ldcg(b.row_slice + row);
            if (NT == 4 && R == 32) {      // 16-byte aligned: one float4 of U, one of w
                const float4 u4 = __ldcg(reinterpret_cast<const float4 *>(U + row * 32 + 4 * g));
                const float4 w4 = __ldcg(reinterpret_cast<const float4 *>(Wf + (int64_t)k * 32 + 4 * g));
                v[p][0] = u4.x * w4.x;
                v[p][1] = u4.y * w4.y;
                v[p][2] = u4.z * w4.z;
                v[p][3] = u4.w * w4.w;
            } else {
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int r = NT * g + nt;
                    if (r < R) v[p][nt] = U[row * R + r] * Wf[(int64_t)k * R + r];
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) m = fmaxf(m, fabsf(v[p][nt]));
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    }
    const int eu = xq_exp(m);
    const float ts = xq_pow2(10 - eu);
    uint32_t *blk = Uf + G * ft_ublk(NT);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        uint4 f;
        xq_split(v[0][nt] * ts, v[1][nt] * ts, f.x, f.z);
        xq_split(v[2][nt] * ts, v[3][nt] * ts, f.y, f.w);
        reinterpret_cast<uint4 *>(blk)[32 * nt + lane] = f;
    }
    if (lane == 0) reinterpret_cast<int4 *>(blk)[32 * NT] = make_int4(ft_xscale_exp(ex), eu, 0, 0);
}

// ---------------------------------------------------------------------------
// k_f_tc: F partials.  CTA (bx, by) takes the general rows
// [bx·rows_per_cta, ...) (rows_per_cta a multiple of 16, so its k-steps are
// k_utilde's groups) and the columns [512·by, 512·by + 512).  Warp w takes
// column group jg = w % njg (64 columns) and the k-steps (16 rows)
// ks ≡ w / njg (mod nrs) of the CTA's rows, njg = column groups of this CTA,
// nrs = FT_WARPS / njg.  A stage holds a k-step's 16 X row segments (64
// columns) and its Ũ fragment block.
//
// MMA orientation: D (16 j × 8 r) += Xᵀ (16 j × 16 rows) · Ũ (16 rows × 8 r).
// Lane (g, tg) holds the k-slots (rows) 2tg, 2tg+1, 2tg+8, 2tg+9 of the
// k-step; for m-tile t its m-slots g and g+8 are columns
// jg0 + 32(t/2) + 4g + 2(t%2) + {0, 1}, so the lane reads each row as two
// float4s (columns jg0 + 4g and jg0 + 32 + 4g); n-slot g of n-tile nt is
// rank column NT·g + nt (the order of k_utilde's fragments).  The k-step's X
// is scaled by 2^sxe, its Ũ comes split and scaled by 2^(10 - eu), and its
// product is scaled back by 2^(eu - 10 - sxe).
constexpr int FT_THREADS = 256;
constexpr int FT_WARPS = FT_THREADS / 32;
constexpr int FT_S = 3;                   // stages per warp ring
constexpr int FT_JCTA = 512;              // columns per CTA (8 groups of 64)
constexpr int FT_XP = 68;                 // floats per staged X row (≡ 4 mod 8: conflict-free)
constexpr int FT_FLUSH = 16;              // k-steps summed in registers before the smem sum

__host__ __device__ constexpr int ft_stage(int NT) { return 16 * FT_XP + ft_ublk(NT); }
// rings, then per warp its FP32 accumulator (512·NT floats), then the barriers
__host__ __device__ inline size_t ft_smem(int NT) {
    return (size_t)FT_WARPS * FT_S * ft_stage(NT) * 4 + (size_t)FT_WARPS * 512 * NT * 4 +
           (size_t)FT_WARPS * FT_S * 8;
}

template <int NT>
__global__ void __launch_bounds__(FT_THREADS, 1)
    k_f_tc(const float *__restrict__ X, BatchDev b, int J, int R, const uint32_t *__restrict__ Uf,
           int64_t rows_per_cta, float *__restrict__ Fpart, int *__restrict__ err,
           unsigned long long *__restrict__ pc) {
    extern __shared__ __align__(16) float ft_sm[];
    constexpr int STG = ft_stage(NT), UB = ft_ublk(NT);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    float *ring = ft_sm + (size_t)warp * FT_S * STG;
    // Two-level sum: FT_FLUSH k-steps in registers, then into the warp's FP32
    // block in shared memory (slot ((t·NT + nt)·4 + e)·32 + lane), so no FP32
    // running sum takes more than a few dozen terms.
    float *wacc = ft_sm + (size_t)FT_WARPS * FT_S * STG + (size_t)warp * 512 * NT;
    uint64_t *bars = reinterpret_cast<uint64_t *>(ft_sm + (size_t)FT_WARPS * FT_S * STG +
                                                  (size_t)FT_WARPS * 512 * NT) + warp * FT_S;
    if (lane == 0) {
        for (int s = 0; s < FT_S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = lane; e < 512 * NT; e += 32) wacc[e] = 0.f;
    __syncwarp();
    const int jc0 = FT_JCTA * blockIdx.y;
    const int jcn = min(FT_JCTA, J - jc0);
    const int njg = (jcn + 63) / 64;
    const int nrs = FT_WARPS / njg;
    const int jg = warp % njg, rs = warp / njg;
    const bool active = rs < nrs;
    const int jg0 = jc0 + 64 * jg;
    const bool c0ok = jg0 + 4 * g < J, c1ok = jg0 + 32 + 4 * g < J;
    const uint32_t xbytes = (uint32_t)min(64, J - jg0) * 4;
    const int64_t run0 = run0_of(b);
    const int64_t gbeg = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t gend = b.N_gen < gbeg + rows_per_cta ? b.N_gen : gbeg + rows_per_cta;
    const int nks = (int)((gend - gbeg + 15) / 16);
    const int my_n = (active && rs < nks) ? (nks - 1 - rs) / nrs + 1 : 0;
    int is = 0;
    int64_t ig0 = gbeg + 16 * rs;             // first row of the next k-step to copy
    auto issue = [&]() {
        if (is >= my_n) return;
        const int s = is % FT_S;
        const int nv = (int)(gend - ig0 < 16 ? gend - ig0 : 16);
        float *st = ring + (size_t)s * STG;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (lane == 0) mbar_expect_tx(&bars[s], (uint32_t)nv * xbytes + (uint32_t)UB * 4);
        __syncwarp();
        if (lane < nv) {
            const int64_t row = gen_row_fast(b, run0, ig0 + lane);
            bulk_g2s(st + lane * FT_XP, X + row * (int64_t)J + jg0, xbytes, &bars[s]);
        }
        if (lane == 31) bulk_g2s(st + 16 * FT_XP, Uf + (ig0 / 16) * UB, (uint32_t)UB * 4, &bars[s]);
        ig0 += 16 * nrs;
        ++is;
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
    const int roff[4] = {2 * tg, 2 * tg + 1, 2 * tg + 8, 2 * tg + 9};
    bool aborted = false;
    int i = 0;
    int64_t cg0 = gbeg + 16 * rs;             // first row of the k-step being computed
    long long cw = 0;                         // profiling: cycles waiting on stages
    const long long c0 = pc ? clock64() : 0;
    for (; i < my_n; ++i) {
        issue();
        const int s = i % FT_S;
        const long long w0 = pc ? clock64() : 0;
        if (!sb_wait(&bars[s], (uint32_t)(i / FT_S) & 1u, err)) {
            aborted = true;
            break;
        }
        if (pc) cw += clock64() - w0;
        const float *st = ring + (size_t)s * STG;
        const uint4 *ub = reinterpret_cast<const uint4 *>(st + 16 * FT_XP);
        const int nv = (int)(gend - cg0 < 16 ? gend - cg0 : 16);
        cg0 += 16 * nrs;
        const int4 sc = *reinterpret_cast<const int4 *>(ub + 32 * NT);
        const float tu = xq_pow2(sc.y - 10) * xq_pow2(-sc.x);
        float4 xv[4][2];
        uint4 bf[NT];                      // {bh0, bh1, bl0, bl1} of n-tile nt
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (nv == 16 && c0ok && c1ok) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float *xr = st + roff[p] * FT_XP + 4 * g;
                xv[p][0] = *reinterpret_cast<const float4 *>(xr);
                xv[p][1] = *reinterpret_cast<const float4 *>(xr + 32);
            }
        } else {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const bool rv = roff[p] < nv;
                const float *xr = st + roff[p] * FT_XP + 4 * g;
                xv[p][0] = (rv && c0ok) ? *reinterpret_cast<const float4 *>(xr) : z;
                xv[p][1] = (rv && c1ok) ? *reinterpret_cast<const float4 *>(xr + 32) : z;
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) bf[nt] = ub[32 * nt + lane];
        __syncwarp();                      // stage s is read: free for its next copy
        {                                  // X scale of the group: 2^sxe
            const float sx = xq_pow2(sc.x);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                xv[p][0] = f4scale(xv[p][0], sx);
                xv[p][1] = f4scale(xv[p][1], sx);
            }
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
            for (int nt = 0; nt < NT; ++nt) {   // main and correction terms apart
                float d[4], dc[4];
                xq_mma0(d, a0h, a1h, a2h, a3h, bf[nt].x, bf[nt].y);
                xq_mma0(dc, a0h, a1h, a2h, a3h, bf[nt].z, bf[nt].w);
                xq_mma(dc, a0l, a1l, a2l, a3l, bf[nt].x, bf[nt].y);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[t][nt][e] = fmaf(d[e] + dc[e], tu, acc[t][nt][e]);
            }
        }
        if ((i + 1) % FT_FLUSH == 0 || i + 1 == my_n) {
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float &w = wacc[((t * NT + nt) * 4 + e) * 32 + lane];
                        w += acc[t][nt][e];
                        acc[t][nt][e] = 0.f;
                    }
        }
    }
    if (aborted) {                         // let the copies already issued land
        for (int k = i; k < is; ++k) sb_wait(&bars[k % FT_S], (uint32_t)(k / FT_S) & 1u, err);
    }
    if (pc && lane == 0) {
        atomicAdd(&pc[0], (unsigned long long)cw);
        atomicAdd(&pc[1], (unsigned long long)(clock64() - c0));
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[t][nt][e] = wacc[((t * NT + nt) * 4 + e) * 32 + lane];
    // warps of one column group (row subgroups 1.., in order) add into row
    // subgroup 0, which writes the CTA's partial; the rings are free now
    float *red_all = ft_sm;
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

// ---------------------------------------------------------------------------
// k_big_b_tc: the chunked path's per-chunk products on the tensor cores (the
// split row pipeline).  One warp per chunk of <= 256 rows of one slice:
//   U = (P'·R_V⁻ᵀ)·S_k⁻¹ (Lemma 1's fast path, Eq. 11), written out;
//   ΔD = UᵀU and Δc = diag(ΔD S_k Γ) (Eqs. 15-16), the chunk's partials.
// Both products use the FP16 split with the main and correction terms in
// separate accumulators, 16 rows at a time: U's tile goes through a padded
// shared block (pitch BT_UP, conflict-free) to become both MMA operands of
// ΔD (A = Uᵀ and B = U read the same values).  Chunks of slices that need
// the general map (a zero weight, or a singular Γ) take big_chunk's SIMT
// path.  R <= 32, R even (8-byte aligned P' and U pairs for the float2 accesses).
constexpr int BT_UP = 36;                 // staged U tile pitch (≡ 4 mod 32 words: 8tg + g banks)

static __global__ void __launch_bounds__(256, 2) k_big_b_tc(FusedArgs a, BigArgs bg) {
    __shared__ __align__(16) float Us[FU_WARPS][32][FU_RP];      // SIMT fallback
    __shared__ __align__(16) float Tw[FU_WARPS][32 * BT_UP];     // U tile / ΔD staging
    __shared__ float Wi_all[FU_WARPS][32];                        // 1/w_k of the chunk's slice
    __shared__ uint4 Mf_all[FU_WARPS][8][32];                     // R_V⁻ᵀ fragments per lane
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    const int R = a.R;
    const unsigned full = 0xffffffffu;
    float *T = Tw[warp];
    float *Wi = Wi_all[warp];
    uint4 (*Mf)[32] = Mf_all[warp];
    const bool gam_ok = *a.gam_ok != 0;
    // R_V⁻ᵀ as B fragments (k = t, n = c), scaled by 2^bm: the same for every
    // chunk of the update (U = (P'·R_V⁻ᵀ) ∘ 1/w_k column by column, so S_k⁻¹
    // is applied to the output columns)
    float mmax = 0.f;
    for (int e0 = 0; e0 < R * R; e0 += 32)
        if (e0 + lane < R * R) mmax = fmaxf(mmax, fabsf(a.GPf[e0 + lane]));
#pragma unroll
    for (int o = 16; o; o >>= 1) mmax = fmaxf(mmax, __shfl_xor_sync(full, mmax, o));
    const int bm = 10 - xq_exp(mmax);
    const float bsc = xq_pow2(bm);
    // {b0hi, b1hi, b0lo, b1lo} of n-tile nt, k-step ks at Mf[2nt + ks][lane]
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c = 8 * nt + g;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = 16 * ks + 2 * tg + (u & 1) + 8 * (u >> 1);
                v[u] = (t < R && c < R) ? a.GPf[t * R + c] * bsc : 0.f;
            }
            uint4 f;
            xq_split(v[0], v[1], f.x, f.z);
            xq_split(v[2], v[3], f.y, f.w);
            Mf[2 * nt + ks][lane] = f;
        }
    }
    for (int ch = blockIdx.x * FU_WARPS + warp; ch < bg.n_chunks; ch += gridDim.x * FU_WARPS) {
        const int k = bg.ch_k[ch];
        const double wold_d = lane < R ? a.W[(int64_t)k * R + lane] : 1.0;
        const bool fast = gam_ok && __all_sync(full, wold_d != 0.0);
        if (!fast) {
            big_chunk(a, bg, ch, Us[warp]);
            continue;
        }
        const int64_t row0 = bg.ch_row0[ch];
        const int n = bg.ch_n[ch];
        __syncwarp();
        Wi[lane] = lane < R ? 1.0f / (float)wold_d : 0.f;   // 1/w_k (zero past R)
        __syncwarp();
        float dd[2][4][4];                        // ΔD in the MMA C layout: [mt][nt][e]
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) dd[mt][nt][e] = 0.f;
        for (int i0 = 0; i0 < n; i0 += 16) {
            const int m = min(16, n - i0);
            const bool va = g < m, vb = g + 8 < m;
            const float *ya = bg.Y + (row0 + i0 + g) * R, *yb = ya + 8 * R;
            // P' A fragments (rows g, g+8; k-slots 2tg, 2tg+1, 2tg+8, 2tg+9)
            float2 p[2][4];
            float pm0 = 0.f, pm1 = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int c0 = 16 * ks + 2 * tg, c1 = c0 + 8;
                const float2 z = make_float2(0.f, 0.f);
                p[ks][0] = (va && c0 < R) ? *reinterpret_cast<const float2 *>(ya + c0) : z;
                p[ks][1] = (vb && c0 < R) ? *reinterpret_cast<const float2 *>(yb + c0) : z;
                p[ks][2] = (va && c1 < R) ? *reinterpret_cast<const float2 *>(ya + c1) : z;
                p[ks][3] = (vb && c1 < R) ? *reinterpret_cast<const float2 *>(yb + c1) : z;
                pm0 = fmaxf(pm0, fmaxf(fmaxf(fabsf(p[ks][0].x), fabsf(p[ks][0].y)),
                                       fmaxf(fabsf(p[ks][2].x), fabsf(p[ks][2].y))));
                pm1 = fmaxf(pm1, fmaxf(fmaxf(fabsf(p[ks][1].x), fabsf(p[ks][1].y)),
                                       fmaxf(fabsf(p[ks][3].x), fabsf(p[ks][3].y))));
            }
            pm0 = fmaxf(pm0, __shfl_xor_sync(full, pm0, 1));
            pm0 = fmaxf(pm0, __shfl_xor_sync(full, pm0, 2));
            pm1 = fmaxf(pm1, __shfl_xor_sync(full, pm1, 1));
            pm1 = fmaxf(pm1, __shfl_xor_sync(full, pm1, 2));
            const int x0 = ft_xscale_exp(xq_exp(pm0)), x1 = ft_xscale_exp(xq_exp(pm1));
            const float s0 = xq_pow2(x0), s1 = xq_pow2(x1);
            float um[4][4], uc[4][4];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) um[nt][e] = uc[nt][e] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t ah[4], al[4];
                xq_split(p[ks][0].x * s0, p[ks][0].y * s0, ah[0], al[0]);
                xq_split(p[ks][1].x * s1, p[ks][1].y * s1, ah[1], al[1]);
                xq_split(p[ks][2].x * s0, p[ks][2].y * s0, ah[2], al[2]);
                xq_split(p[ks][3].x * s1, p[ks][3].y * s1, ah[3], al[3]);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const uint4 f = Mf[2 * nt + ks][lane];
                    xq_mma(um[nt], ah[0], ah[1], ah[2], ah[3], f.x, f.y);
                    xq_mma(uc[nt], ah[0], ah[1], ah[2], ah[3], f.z, f.w);
                    xq_mma(uc[nt], al[0], al[1], al[2], al[3], f.x, f.y);
                }
            }
            // U rows: scale back (row scale and M's 2^bm), write out, stage in T
            const float r0s = xq_pow2(-x0) * xq_pow2(-bm), r1s = xq_pow2(-x1) * xq_pow2(-bm);
            __syncwarp();
            float umax = 0.f;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = 8 * nt + 2 * tg;
                const float w0 = Wi[c], w1 = Wi[c + 1];
                const float u00 = (um[nt][0] + uc[nt][0]) * r0s * w0;
                const float u01 = (um[nt][1] + uc[nt][1]) * r0s * w1;
                const float u10 = (um[nt][2] + uc[nt][2]) * r1s * w0;
                const float u11 = (um[nt][3] + uc[nt][3]) * r1s * w1;
                const bool cv = c < R;
                T[g * BT_UP + c] = (va && cv) ? u00 : 0.f;
                T[g * BT_UP + c + 1] = (va && cv) ? u01 : 0.f;
                T[(g + 8) * BT_UP + c] = (vb && cv) ? u10 : 0.f;
                T[(g + 8) * BT_UP + c + 1] = (vb && cv) ? u11 : 0.f;
                if (va && cv) *reinterpret_cast<float2 *>(a.U + (row0 + i0 + g) * R + c) = make_float2(u00, u01);
                if (vb && cv) *reinterpret_cast<float2 *>(a.U + (row0 + i0 + g + 8) * R + c) = make_float2(u10, u11);
                if (va && cv) umax = fmaxf(umax, fmaxf(fabsf(u00), fabsf(u01)));
                if (vb && cv) umax = fmaxf(umax, fmaxf(fabsf(u10), fabsf(u11)));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(full, umax, o));
            const int eu = xq_exp(umax);
            const float su = xq_pow2(10 - eu);
            __syncwarp();
            // ΔD += UᵀU for this tile: u(row, col) pairs at rows 2tg, 2tg+1 (b0)
            // and 2tg+8, 2tg+9 (b1), column 8nt + g; A = Uᵀ's fragments for
            // m-tile mt are those of n-tiles 2mt, 2mt+1
            uint32_t bh[4][2], bl[4][2];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = 8 * nt + g;
                xq_split(T[(2 * tg) * BT_UP + c] * su, T[(2 * tg + 1) * BT_UP + c] * su, bh[nt][0], bl[nt][0]);
                xq_split(T[(2 * tg + 8) * BT_UP + c] * su, T[(2 * tg + 9) * BT_UP + c] * su, bh[nt][1], bl[nt][1]);
            }
            const float uu = xq_pow2(eu - 10) * xq_pow2(eu - 10);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    float d[4], dc[4];
                    xq_mma0(d, bh[2 * mt][0], bh[2 * mt + 1][0], bh[2 * mt][1], bh[2 * mt + 1][1],
                            bh[nt][0], bh[nt][1]);
                    xq_mma0(dc, bh[2 * mt][0], bh[2 * mt + 1][0], bh[2 * mt][1], bh[2 * mt + 1][1],
                            bl[nt][0], bl[nt][1]);
                    xq_mma(dc, bl[2 * mt][0], bl[2 * mt + 1][0], bl[2 * mt][1], bl[2 * mt + 1][1],
                           bh[nt][0], bh[nt][1]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) dd[mt][nt][e] = fmaf(d[e] + dc[e], uu, dd[mt][nt][e]);
                }
            }
        }
        // ΔD (C layout: row 16mt + g (+8), column 8nt + 2tg (+1)) → staging,
        // then Δc = diag(ΔD S Γ) with lane = row, and the chunk's partials
        __syncwarp();
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int r = 16 * mt + g, c = 8 * nt + 2 * tg;
                T[r * 33 + c] = dd[mt][nt][0];
                T[r * 33 + c + 1] = dd[mt][nt][1];
                T[(r + 8) * 33 + c] = dd[mt][nt][2];
                T[(r + 8) * 33 + c + 1] = dd[mt][nt][3];
            }
        __syncwarp();
        const bool act = lane < R;
        const float wl = act ? (float)wold_d : 0.f;
        float sacc = 0.f;
        float *out = bg.dpart + (size_t)ch * (R * R + R);
#pragma unroll 4
        for (int q = 0; q < R; ++q) {
            const float wq = __shfl_sync(full, wl, q);
            // ΔD is symmetric; the MMA's two halves may differ in the last bit
            const float dq = 0.5f * (T[q * 33 + lane] + T[lane * 33 + q]);
            if (act) {
                sacc = fmaf(dq * wq, a.Gdf[q * R + lane].hi, sacc);   // (float)Γ
                out[q * R + lane] = dq;
            }
        }
        if (act) out[R * R + lane] = sacc;
        __syncwarp();
    }
}

}  // namespace dash
