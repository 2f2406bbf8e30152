// Streaming X·Q_V on the Blackwell tensor cores (P3 of a mode-P update,
// Theorem 1's X_k,new V term in the V = Q_V R_V basis):
//
//   k_qv_tf32  Q_V split into TF32 big + small parts, written in the
//              128-byte-swizzled K-major layout the MMA reads (one 8 KB slab
//              per 32 columns of X: rows 0-31 the big parts of Q_V's 32 rank
//              columns, rows 32-63 the small parts; zero past J or R)
//   k_xq_umma  P' = X·Q_V for every general row, the ‖X‖² partials and each
//              row's max-|x| exponent
//   k_utilde_tf32  Ũ = U ∘ w_k,new (the U_k,new S_k,new of Eq. 20) split
//              into TF32 big + small parts, per 32-row block in the
//              swizzled K-major layout of the F pass's B operand
//   k_f_umma   per-chunk partials of F_inc = Σ_rows X(i,:)ᵀ Ũ(i,:) (P5,
//              Eq. 20) on tcgen05 MMAs, A = Xᵀ from tensor memory
//
// Products.  x = big(x) + small(x), big(x) the TF32 value the tensor core
// takes from x's FP32 bits and small(x) = x − big(x) exactly in FP32; Q_V
// likewise.  P' = big(X)·big(Q_V) + big(X)·small(Q_V) + small(X)·big(Q_V)
// (the 3-term TF32 split), each product exact in FP32.  Every 32-column
// stage (4 MMA k-steps) accumulates into a fresh tensor-memory accumulator,
// the main term in its columns 0-31 and the two correction terms in 32-63;
// the epilogue adds main + correction and sums the stages in FP32 registers
// (rounded to nearest).  The tensor core's own accumulation does not round
// to nearest, and over all 64 k-steps of a 512-column row a sum with
// cancelling terms lost ~30× more than the FP16-split kernel; over 4 k-steps
// it stays below that kernel's error.  TF32 keeps FP32's exponent range, so
// no operand needs scaling.
//
// Kernel structure (one persistent CTA per SM, 18 warps, tiles of 128 rows):
//   warp 0     TMA producer: Q_V's slabs once, then per tile and 32-column
//              stage one 128×32 FP32 box of X (SWIZZLE_128B) into a ring of
//              nst stages, each completing on full[s]
//   warp 1     MMA issuer: per stage 4 k-steps of 8 columns, each one
//              M=128 N=64 MMA of big(X) (shared memory) against Q_V's big and
//              small rows and one M=128 N=32 MMA of small(X) (tensor memory)
//              against Q_V's big rows, into accumulator i mod XU_NACC; its
//              commits free the stage (empty[s]) and publish the
//              accumulator (accf[a])
//   warps 2-9  converters, two groups of four taking alternate stages:
//              thread = row of the tile (its TMEM lane); reads its row's 32
//              floats of the stage, writes small(x) into the stage's
//              tensor-memory slot, sums x²
//   warps 10-17 epilogue, two groups of four taking alternate stages: per
//              stage, reads the accumulator (freeing it through acce[a]) and
//              adds it to the row's FP32 sums; at a tile's end the second
//              group hands its sums to the first through tensor memory, which
//              adds them (fixed order) and writes the P' rows
// Two groups per role give each converter and epilogue thread two stage
// times for its chain of shared-memory loads, tensor-memory stores or loads
// and their waits.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dash_kernels_p.cuh"
#include "dash_kernels_stream.cuh"
#include "dash_umma.cuh"

namespace dash {

constexpr int XU_THREADS = 576;
constexpr int XU_SLAB_BYTES = 64 * 128;      // one Q_V slab: 64 rows × 32 floats
constexpr int XU_STAGE_BYTES = 128 * 128;    // one X box: 128 rows × 32 floats
constexpr int XU_TMEM_COLS = 512;            // accumulators 0-255, small(X) slots 256-447, hand-over 480
constexpr int XU_NACC = 4;                   // accumulator ring (64 columns each)
constexpr int XU_MAX_STAGES = 6;             // small(X) slots: 256 + 6·32 <= 448
constexpr uint32_t XU_HAND_COL = 480;        // epilogue hand-over columns 480-511

// big(x): the TF32 value the tensor core uses for an FP32 operand x (its
// 13 low mantissa bits dropped).  small(x) = x − big(x) is exact in FP32.
__device__ __forceinline__ float tf32_big(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Dynamic shared memory of k_xq_umma for J columns and nst stages:
// alignment slack, the Q_V slabs, the X ring, barriers and scratch.
__host__ __device__ inline size_t xu_smem(int J, int nst) {
    const int nslab = (J + 31) / 32;
    return 1024 + (size_t)nslab * XU_SLAB_BYTES + (size_t)nst * XU_STAGE_BYTES + 512;
}
// Largest ring depth that fits the 227 KB per-CTA limit (0: does not fit).
inline int xu_stages(int J) {
    const size_t cap = 232448;
    for (int nst = XU_MAX_STAGES; nst >= 3; --nst)
        if (xu_smem(J, nst) <= cap) return nst;
    return 0;
}

// Q_V (J×R FP32 row-major) into nslab swizzled slabs (see above).
static __global__ void k_qv_tf32(const float *__restrict__ QV, int J, int R, float *__restrict__ out) {
    const int nslab = (J + 31) / 32;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;      // (slab, row, k)
    if (i >= nslab * 64 * 32) return;
    const int sl = i / 2048, n = (i / 32) % 64, kc = i % 32;
    const int j = 32 * sl + kc, r = n & 31;
    float v = 0.f;
    if (j < J && r < R) {
        const float q = QV[(int64_t)j * R + r];
        const float big = tf32_big(q);
        v = n < 32 ? big : q - big;
    }
    reinterpret_cast<float *>(reinterpret_cast<char *>(out) + (size_t)sl * XU_SLAB_BYTES + umma::swz(n, kc))[0] = v;
}

struct XuArgs {
    const float *qv_slabs;   // k_qv_tf32 output
    float *P;                // P' rows, N×R FP32 (row row0 + g for general row g)
    double *xn_part;         // per-CTA Σ‖x‖²
    int *err;                // [0]: timed-out waits, [3]: update abandoned
    int64_t N_gen;           // rows (the tensor map's outer extent)
    int64_t row0;            // batch row of general row 0
    int J, R, nst;
    long long wait_limit;    // cycles before a wait gives up
    int skip_first_copy;     // test hook: CTA 0 never issues its first stage's copy
    unsigned long long *pc;  // optional: cycles waiting per role, and per CTA in total
};

// Clock of this thread when profiling, else 0.
__device__ __forceinline__ long long xu_clk(const unsigned long long *pc) { return pc ? clock64() : 0; }

static __global__ void __launch_bounds__(XU_THREADS, 1)
    k_xq_umma(const __grid_constant__ CUtensorMap tmX, XuArgs a) {
    extern __shared__ uint8_t xu_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(xu_raw) + 1023) & ~(uintptr_t)1023);
    const int nslab = (a.J + 31) / 32, nst = a.nst;
    uint8_t *sB = sm;
    uint8_t *sX = sm + (size_t)nslab * XU_SLAB_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sX + (size_t)nst * XU_STAGE_BYTES);
    uint64_t *conv = full + nst, *empty = conv + nst;
    uint64_t *accf = empty + nst, *acce = accf + XU_NACC, *bfull = acce + XU_NACC, *done = bfull + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
    double *red = reinterpret_cast<double *>(tslot + 2);      // 8 converter warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = (a.N_gen + 127) / 128;
    const int my_nt = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int total = my_nt * nslab;
    const long long c_start = xu_clk(a.pc);
    long long c_wait = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 4);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < XU_NACC; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(bfull, 1);
        mbar_init(done, 1);
        *abort_f = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, XU_TMEM_COLS);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *tslot;
    if (warp == 0) {
        // ---- TMA producer ----
        if (lane == 0) {
            mbar_expect_tx(bfull, (uint32_t)nslab * XU_SLAB_BYTES);
            for (int sl = 0; sl < nslab; ++sl)
                bulk_g2s(sB + (size_t)sl * XU_SLAB_BYTES, a.qv_slabs + (size_t)sl * (XU_SLAB_BYTES / 4),
                         XU_SLAB_BYTES, bfull);
            int issued = 0;
            for (int it = 0; it < total; ++it) {
                const int s = it % nst, u = it / nst;
                const long long w0 = xu_clk(a.pc);
                if (u > 0 && !umma::wait_or_abort(&empty[s], (uint32_t)(u - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                c_wait += xu_clk(a.pc) - w0;
                const int64_t tile = blockIdx.x + (int64_t)(it / nslab) * gridDim.x;
                mbar_expect_tx(&full[s], XU_STAGE_BYTES);
                if (!(a.skip_first_copy && blockIdx.x == 0 && it == 0))
                    umma::tma_load_2d(sX + (size_t)s * XU_STAGE_BYTES, &tmX, 32 * (it % nslab),
                                      (int)(tile * 128), &full[s]);
                ++issued;
            }
            // copies still in flight land before the CTA exits: the last use
            // of each stage is the newest phase its barrier can complete
            for (int it = issued - 1; it >= 0 && it >= issued - nst; --it) {
                const int s = it % nst, u = it / nst;
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s], (uint32_t)u & 1u) && clock64() - t0 < a.wait_limit) {
                }
            }
            const long long t0 = clock64();
            while (!mbar_try_wait(bfull, 0) && clock64() - t0 < a.wait_limit) {
            }
            if (a.pc) atomicAdd(&a.pc[0], (unsigned long long)c_wait);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0 && total > 0 && umma::wait_or_abort(bfull, 0, abort_f, a.err, a.wait_limit)) {
            umma::fence_after();
            constexpr uint32_t id64 = umma::idesc_tf32(128, 64, 0, 0);
            constexpr uint32_t id32 = umma::idesc_tf32(128, 32, 0, 0);
            const uint32_t sx0 = smem_u32(sX), sb0 = smem_u32(sB);
            for (int it = 0; it < total; ++it) {
                const int s = it % nst, u = it / nst;
                const int kk = it % nslab;
                const int ab = it % XU_NACC, v = it / XU_NACC;
                const long long w0 = xu_clk(a.pc);
                if (v > 0 && !umma::wait_or_abort(&acce[ab], (uint32_t)(v - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                if (!umma::wait_or_abort(&conv[s], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit)) break;
                c_wait += xu_clk(a.pc) - w0;
                umma::fence_after();
                const uint32_t dcol = tmem + (uint32_t)ab * 64u;
                const uint32_t acol = tmem + 256u + (uint32_t)s * 32u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint64_t ad = umma::sdesc_sw128(sx0 + (uint32_t)s * XU_STAGE_BYTES + 32u * k, 16, 1024);
                    const uint64_t bd = umma::sdesc_sw128(sb0 + (uint32_t)kk * XU_SLAB_BYTES + 32u * k, 16, 1024);
                    umma::mma_ss(dcol, ad, bd, id64, k != 0);
                    umma::mma_ts(dcol + 32u, acol + 8u * k, bd, id32, 1u);
                }
                umma::commit(&empty[s]);
                umma::commit(&accf[ab]);
            }
            // every MMA issued has completed before the tensor memory is freed
            umma::commit(done);
            const long long t0 = clock64();
            while (!mbar_try_wait(done, 0) && clock64() - t0 < a.wait_limit) {
            }
            if (a.pc) atomicAdd(&a.pc[1], (unsigned long long)c_wait);
        }
    } else if (warp < 10) {
        // ---- converters: group gr takes stages it ≡ gr (mod 2); thread = tile
        // row r, TMEM lane r ----
        const int q = warp & 3, gr = (warp - 2) >> 2, r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        double xn = 0.0;
        for (int it = gr; it < total; it += 2) {
            const int s = it % nst, u = it / nst;
            const long long w0 = xu_clk(a.pc);
            const bool ok = umma::wait_or_abort(&full[s], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) break;
            c_wait += xu_clk(a.pc) - w0;
            const uint8_t *row = sX + (size_t)s * XU_STAGE_BYTES + (size_t)r * 128;
            uint32_t sv[32];
            float xs = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4) {
                const float4 x = *reinterpret_cast<const float4 *>(row + ((c4 ^ (r & 7)) << 4));
                const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    xs = fmaf(xv[e], xv[e], xs);
                    sv[4 * c4 + e] = __float_as_uint(xv[e] - tf32_big(xv[e]));
                }
            }
            umma::tmem_st32(lane_base + 256u + (uint32_t)s * 32u, sv);
            xn += (double)xs;
            umma::tmem_st_wait();
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&conv[s]);
        }
        xn = warp_sum(xn);
        if (lane == 0) red[warp - 2] = xn;
        if (a.pc && lane == 0) atomicAdd(&a.pc[2], (unsigned long long)c_wait);
    } else {
        // ---- epilogue: group gr takes stages it ≡ gr (mod 2); thread = tile
        // row r.  Every thread runs the same hand-over barriers per tile, also
        // after an abort (then without waiting or touching tensor memory). ----
        const int q = warp & 3, gr = (warp - 10) >> 2, r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        bool dead = false;
        for (int tc = 0; tc < my_nt; ++tc) {
            float acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
            for (int kk = 0; kk < nslab; ++kk) {
                const int it = tc * nslab + kk;
                if ((it & 1) != gr || dead) continue;
                const int ab = it % XU_NACC, v = it / XU_NACC;
                const long long w0 = xu_clk(a.pc);
                const bool ok = umma::wait_or_abort(&accf[ab], (uint32_t)v & 1u, abort_f, a.err, a.wait_limit);
                if (!__all_sync(0xffffffffu, ok)) {
                    dead = true;
                    continue;
                }
                c_wait += xu_clk(a.pc) - w0;
                umma::fence_after();
                uint32_t t[32];
                umma::tmem_ld32(lane_base + (uint32_t)ab * 64u, t);
                umma::tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 32; ++c) acc[c] += __uint_as_float(t[c]);
                umma::tmem_ld32(lane_base + (uint32_t)ab * 64u + 32u, t);
                umma::tmem_ld_wait();
                umma::fence_before();
                __syncwarp();
                if (lane == 0) umma::mbar_arrive(&acce[ab]);
#pragma unroll
                for (int c = 0; c < 32; ++c) acc[c] += __uint_as_float(t[c]);
            }
            // hand-over: group 1's sums to group 0 through tensor memory
            if (gr == 1 && !dead) {
                uint32_t t[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) t[c] = __float_as_uint(acc[c]);
                umma::tmem_st32(lane_base + XU_HAND_COL, t);
                umma::tmem_st_wait();
            }
            umma::fence_before();
            asm volatile("bar.sync 1, 256;" ::: "memory");
            umma::fence_after();
            if (gr == 0 && !dead) {
                uint32_t t[32];
                umma::tmem_ld32(lane_base + XU_HAND_COL, t);
                umma::tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 32; ++c) acc[c] += __uint_as_float(t[c]);
                const int64_t g = (blockIdx.x + (int64_t)tc * gridDim.x) * 128 + r;
                if (g < a.N_gen) {
                    float *p = a.P + (a.row0 + g) * a.R;
                    if ((a.R & 3) == 0) {
#pragma unroll
                        for (int c = 0; c < 32; c += 4)
                            if (c < a.R)
                                *reinterpret_cast<float4 *>(p + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (c < a.R) p[c] = acc[c];
                    }
                }
            }
            umma::fence_before();
            asm volatile("bar.sync 2, 256;" ::: "memory");
            umma::fence_after();
        }
        if (a.pc && lane == 0) atomicAdd(&a.pc[3], (unsigned long long)c_wait);
    }
    umma::fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int q = 0; q < 8; ++q) sum += red[q];
        a.xn_part[blockIdx.x] = sum;
        if (a.pc) atomicAdd(&a.pc[4], (unsigned long long)(clock64() - c_start));
    }
    if (warp == 0) {
        umma::fence_after();
        umma::tmem_free(tmem, XU_TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// The F pass (Eq. 20's new term).  The contraction runs over rows, which are
// the strided index of X, so X enters as A = Xᵀ held in tensor memory (lane =
// column j of the CTA's 128-column tile, TMEM column = row), written there by
// converter warps that read each staged row block column by column; B = Ũᵀ
// (rank columns as MMA N, rows as K) comes from k_utilde_tf32 already split
// and swizzled.  Per 32-row stage and k-step of 8 rows:
//   D[:, 0:64]  (+)= big(X)ᵀ · [big(Ũ) | small(Ũ)]     (M=128, N=64)
//   D[:, 32:64]  += small(X)ᵀ · big(Ũ)                   (M=128, N=32)
// Every stage accumulates into a fresh accumulator of a ring of FB_NACC in
// tensor memory (4 k-steps each), which the epilogue warps add to FP32
// register sums (main + correction added in FP32, rounded to nearest): the
// same split of the sum as the X·Q_V pass.
constexpr int FB_THREADS = 320;
constexpr int FB_XSTAGE = 32 * 128 * 4;        // 32 rows × 128 columns of X
constexpr int FB_UBLK = 64 * 128;              // Ũ block: 64 rank rows × 32 rows
constexpr int FB_STAGE = FB_XSTAGE + FB_UBLK;
constexpr int FB_NST = 4;
constexpr int FB_NACC = 4;
constexpr int FB_TMEM_COLS = 512;              // accumulators 0-255, A slots from 256 (64 each)

__host__ __device__ inline size_t fb_smem() { return 1024 + (size_t)FB_NST * FB_STAGE + 512; }

// Ũ(g, r) = U(row(g), r)·w_k,new(r) (FP32 product with the FP32 copy of the
// new weights) for general rows g, split into big + small and written per
// 32-row block G at Ub + G·FB_UBLK: rank row r (big) and 32 + r (small), K
// position g mod 32, 128-byte swizzled.  Rows past N_gen and ranks past R
// are zero.  One CTA of 256 threads per block.
static __global__ void __launch_bounds__(256) k_utilde_tf32(BatchDev b, int R, const float *__restrict__ U,
                                                           const float *__restrict__ Wf, float *__restrict__ Ub) {
    __shared__ float t[32][33];
    const int64_t G = blockIdx.x;
    const int64_t run0 = run0_of(b);
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int i = e / 32, r = e % 32;           // row in block, rank column
        const int64_t g = 32 * G + i;
        float v = 0.f;
        if (g < b.N_gen && r < R) {
            const int64_t row = gen_row_fast(b, run0, g);
            const int k = __ldcg(b.row_slice + row);
            v = __ldcg(U + row * R + r) * __ldcg(Wf + (int64_t)k * R + r);
        }
        t[i][r] = v;
    }
    __syncthreads();
    char *blk = reinterpret_cast<char *>(Ub) + (size_t)G * FB_UBLK;
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
        const int n = e / 32, i = e % 32;           // rank row of the block, row in block
        const float u = t[i][n & 31];
        const float big = tf32_big(u);
        *reinterpret_cast<float *>(blk + umma::swz(n, i)) = n < 32 ? big : u - big;
    }
}

struct FbArgs {
    const float *Ub;         // k_utilde_tf32 blocks
    float *Fpart;            // per row chunk: J×R FP32 partial
    int *err;
    int64_t N_gen;
    int64_t rows_per_cta;    // a multiple of 32
    int J, R;
    long long wait_limit;
};

// CTA (c, t): rows [c·rows_per_cta, ...) of the general rows, columns
// [128t, 128t + 128).  Warps: 0 producer (TMA box of 32 rows × 128 columns,
// no swizzle, plus the Ũ block by bulk copy), 1 MMA issuer, 2-5 converters
// (thread = column j = TMEM lane), 6-9 epilogue (thread = column j).
static __global__ void __launch_bounds__(FB_THREADS, 1)
    k_f_umma(const __grid_constant__ CUtensorMap tmX, FbArgs a) {
    extern __shared__ uint8_t fb_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(fb_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + (size_t)FB_NST * FB_STAGE);
    uint64_t *conv = full + FB_NST, *empty = conv + FB_NST;
    uint64_t *accf = empty + FB_NST, *acce = accf + FB_NACC, *done = acce + FB_NACC;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g0 = (int64_t)blockIdx.x * a.rows_per_cta;
    const int64_t g1 = min(a.N_gen, g0 + a.rows_per_cta);
    const int nstage = g1 > g0 ? (int)((g1 - g0 + 31) / 32) : 0;
    const int j0 = 128 * blockIdx.y;
    if (threadIdx.x == 0) {
        for (int s = 0; s < FB_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 4);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < FB_NACC; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(done, 1);
        *abort_f = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma::tmem_alloc(tslot, FB_TMEM_COLS);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *tslot;
    if (warp == 0) {
        // ---- producer ----
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nstage; ++i) {
                const int s = i % FB_NST, u = i / FB_NST;
                if (u > 0 && !umma::wait_or_abort(&empty[s], (uint32_t)(u - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                uint8_t *st = sm + (size_t)s * FB_STAGE;
                mbar_expect_tx(&full[s], FB_STAGE);
                umma::tma_load_2d(st, &tmX, j0, (int)(g0 + 32 * i), &full[s]);
                bulk_g2s(st + FB_XSTAGE, a.Ub + (size_t)(g0 / 32 + i) * (FB_UBLK / 4), FB_UBLK, &full[s]);
                ++issued;
            }
            for (int i = issued - 1; i >= 0 && i >= issued - FB_NST; --i) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[i % FB_NST], (uint32_t)(i / FB_NST) & 1u) && clock64() - t0 < a.wait_limit) {
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0 && nstage > 0) {
            constexpr uint32_t id64 = umma::idesc_tf32(128, 64, 0, 0);
            constexpr uint32_t id32 = umma::idesc_tf32(128, 32, 0, 0);
            const uint32_t s0 = smem_u32(sm);
            for (int i = 0; i < nstage; ++i) {
                const int s = i % FB_NST, u = i / FB_NST;
                const int ab = i % FB_NACC, v = i / FB_NACC;
                if (v > 0 && !umma::wait_or_abort(&acce[ab], (uint32_t)(v - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                if (!umma::wait_or_abort(&conv[s], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit)) break;
                umma::fence_after();
                const uint32_t dcol = tmem + (uint32_t)ab * 64u;
                const uint32_t abig = tmem + 256u + (uint32_t)s * 64u;
                const uint32_t ub = s0 + (uint32_t)s * FB_STAGE + FB_XSTAGE;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint64_t bd = umma::sdesc_sw128(ub + 32u * k, 16, 1024);
                    umma::mma_ts(dcol, abig + 8u * k, bd, id64, k != 0);
                    umma::mma_ts(dcol + 32u, abig + 32u + 8u * k, bd, id32, 1u);
                }
                umma::commit(&empty[s]);
                umma::commit(&accf[ab]);
            }
            umma::commit(done);
            const long long t0 = clock64();
            while (!mbar_try_wait(done, 0) && clock64() - t0 < a.wait_limit) {
            }
        }
    } else if (warp < 6) {
        // ---- converters: thread = column jl of the tile (TMEM lane jl) ----
        const int q = warp & 3, jl = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        for (int i = 0; i < nstage; ++i) {
            const int s = i % FB_NST, u = i / FB_NST;
            const bool ok = umma::wait_or_abort(&full[s], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) break;
            const float *xs = reinterpret_cast<const float *>(sm + (size_t)s * FB_STAGE) + jl;
            uint32_t bg[32], sl[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const float x = xs[r * 128];
                const float big = tf32_big(x);
                bg[r] = __float_as_uint(big);
                sl[r] = __float_as_uint(x - big);
            }
            umma::tmem_st32(lane_base + 256u + (uint32_t)s * 64u, bg);
            umma::tmem_st32(lane_base + 256u + (uint32_t)s * 64u + 32u, sl);
            umma::tmem_st_wait();
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&conv[s]);
        }
    } else {
        // ---- epilogue: thread = column jl ----
        const int q = warp & 3, jl = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        float acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = 0.f;
        bool ok_all = true;
        for (int i = 0; i < nstage; ++i) {
            const int ab = i % FB_NACC, v = i / FB_NACC;
            const bool ok = umma::wait_or_abort(&accf[ab], (uint32_t)v & 1u, abort_f, a.err, a.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) {
                ok_all = false;
                break;
            }
            umma::fence_after();
            uint32_t mn[32], cr[32];
            umma::tmem_ld32(lane_base + (uint32_t)ab * 64u, mn);
            umma::tmem_ld32(lane_base + (uint32_t)ab * 64u + 32u, cr);
            umma::tmem_ld_wait();
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&acce[ab]);
#pragma unroll
            for (int r = 0; r < 32; ++r) acc[r] += __uint_as_float(mn[r]) + __uint_as_float(cr[r]);
        }
        const int j = j0 + jl;
        if (ok_all && j < a.J) {
            float *out = a.Fpart + (int64_t)blockIdx.x * a.J * a.R + (int64_t)j * a.R;
#pragma unroll
            for (int r = 0; r < 32; ++r)
                if (r < a.R) out[r] = acc[r];
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after();
        umma::tmem_free(tmem, FB_TMEM_COLS);
    }
}

}  // namespace dash
