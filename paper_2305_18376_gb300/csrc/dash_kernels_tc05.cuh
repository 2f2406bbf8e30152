// Streaming X·Q_V on the Blackwell tensor cores (P3 of a mode-P update,
// Theorem 1's X_k,new V term in the V = Q_V R_V basis):
//
//   k_qv_tf32  Q_V split into TF32 big + small parts, written in the
//              128-byte-swizzled K-major layout the MMA reads (one 8 KB slab
//              per 32 columns of X: rows 0-31 the big parts of Q_V's 32 rank
//              columns, rows 32-63 the small parts; zero past J or R)
//   k_xq_umma  P' = X·Q_V for every general row, the ‖X‖² partials and each
//              row's max-|x| exponent
//   k_f_umma   per-chunk partials of F_inc = Σ_rows X(i,:)ᵀ Ũ(i,:) (P5,
//              Eq. 20) on tcgen05 MMAs, A = Xᵀ from tensor memory, B = Ũ =
//              U ∘ w_k,new (the U_k,new S_k,new of Eq. 20) built per stage in
//              shared memory from U and the new weights
//
// Products.  x = big(x) + small(x) + O(2^-22 x): big(x) the TF32 value the
// tensor core takes from x's FP32 bits in shared memory (truncation), small(x)
// = x − big(x) rounded to TF32; Q_V with both parts rounded to the nearest
// TF32 value (2^-23).  (Rounding big(x) in place as well measured no gain in
// accuracy and cost 8 % of the pass.)  P' = big(X)·big(Q_V) + big(X)·small(Q_V) + small(X)·big(Q_V)
// (the 3-term TF32 split), each product exact in FP32.  Every 32-column box
// of a stage (4 MMA k-steps) accumulates into a fresh tensor-memory
// accumulator, the main term in its columns 0-31 and the two correction
// terms in 32-63; the epilogue adds them and sums in FP32 registers (rounded
// to nearest).  The tensor core's own accumulation does not round to
// nearest: over all 64 k-steps of a 512-column row a sum with cancelling
// terms lost ~30× more than the FP16-split kernel.  TF32 keeps FP32's exponent range, so
// no operand needs scaling.
//
// Kernel structure (one persistent CTA per SM, 14 warps, tiles of 128 rows):
//   warp 0     TMA producer: per tile and 64-column stage, two 128×32 FP32
//              boxes of X (SWIZZLE_128B) and the stage's two Q_V slabs (from
//              L2; holding all of Q_V would leave room for too few stages)
//              into a ring of nst stages, each completing on full[s] (32 KB
//              of X per stage: a CTA turns its ring over at most ~2 M stages
//              per second, so 16 KB stages would cap a pass near 4.8 TB/s)
//   warp 1     MMA issuer: per stage 8 k-steps of 8 columns, each one
//              M=128 N=64 MMA of big(X) (shared memory) against Q_V's big and
//              small rows and one M=128 N=32 MMA of small(X) (tensor memory)
//              against Q_V's big rows, into accumulator i mod XU_NACC; its
//              commits free the stage (empty[s]) and publish the
//              accumulator (accf[a])
//   warps 2-9  converters (XU_CONV_GROUPS groups of four taking alternate
//              stages): thread = row of the tile (its TMEM lane); reads its
//              row's 64 floats of the stage, writes small(x) into the stage's
//              tensor-memory slot, sums x²
//   warps 10-13 epilogue (XU_EPI_GROUPS groups of four taking alternate
//              stages): per stage, reads the accumulator (freeing it through
//              acce[a]) and adds it to the row's FP32 sums; after a tile's
//              last stage writes the P' rows.  With two groups, the second
//              hands its sums to the first through tensor memory at a tile's
//              end, which adds them in a fixed order.
// More than one group per role gives each thread several stage times for its
// chain of loads, tensor-memory accesses and waits, at the price of
// registers (the whole CTA shares 64 K of them).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dash_kernels_p.cuh"
#include "dash_kernels_stream.cuh"
#include "dash_umma.cuh"

namespace dash {

constexpr int XU_CONV_GROUPS = 2;            // converter groups (alternate stages)
constexpr int XU_EPI_GROUPS = 1;             // epilogue groups (alternate stages)
constexpr int XU_CONV_W0 = 2, XU_EPI_W0 = XU_CONV_W0 + 4 * XU_CONV_GROUPS;
constexpr int XU_THREADS = 32 * (XU_EPI_W0 + 4 * XU_EPI_GROUPS);
constexpr int XU_SLAB_BYTES = 64 * 128;      // one Q_V slab: 64 rows × 32 floats
constexpr int XU_BOX_BYTES = 128 * 128;      // one X box: 128 rows × 32 floats
constexpr int XU_XBYTES = 2 * XU_BOX_BYTES;  // a stage's X: two boxes, 64 columns
constexpr int XU_STAGE_BYTES = XU_XBYTES + 2 * XU_SLAB_BYTES;   // plus its two Q_V slabs
constexpr int XU_TMEM_COLS = 512;            // accumulators 0-255, small(X) slots 256-511
constexpr int XU_NACC = 2;                   // accumulator ring: 128 columns per stage, one
                                             // 64-column accumulator per 32-column box
constexpr int XU_MAX_STAGES = 4;             // small(X) slots of 64 columns: 256 + 4·64 = 512
constexpr uint32_t XU_HAND_COL = 480;        // epilogue hand-over (two epilogue groups only;
                                             // then at most 3 stages)
// A group that takes every G-th stage must always wait on the same ring slots:
// an mbarrier parity wait cannot tell phase u from phase u − 2, so a group
// reaching a slot two phases ahead of its barrier would pass at once.  Ring
// depths are therefore multiples of the group counts.
static_assert(XU_MAX_STAGES % XU_CONV_GROUPS == 0, "converter groups must divide the stage ring");
static_assert(XU_NACC % XU_EPI_GROUPS == 0, "epilogue groups must divide the accumulator ring");
static_assert(XU_EPI_GROUPS == 1 || 256 + XU_MAX_STAGES * 64 <= (int)XU_HAND_COL,
              "the hand-over columns must not overlap the small(X) slots");

// tf32_trunc(x): the TF32 value the tensor core takes from an FP32 operand x
// held in memory (its 13 low mantissa bits dropped).  tf32_rn(x): x rounded
// to the nearest TF32 value (ties away from zero), which the tensor core then
// reads unchanged.  A split x = big + small with small = tf32_rn(x − big)
// keeps x to 2^-22 relative (2^-23 when big = tf32_rn(x) too); a truncated
// small part would keep only 2^-21.
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ float tf32_rn(float x) {
    // round the magnitude at bit 13, half away from zero (the rounding of
    // cvt.rna.tf32.f32), in two integer operations on the full-rate ALU; a
    // carry out of the mantissa moves into the exponent, as it should
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Q_V slabs of J columns: one per 32 columns, rounded up to whole stages of
// two slabs (the slab past J is zero).
__host__ __device__ inline int xu_slabs(int J) { return ((J + 63) / 64) * 2; }
// Dynamic shared memory of k_xq_umma for nst stages (each its X boxes and the
// two Q_V slabs they multiply, which come from L2 again for every tile):
// alignment slack, the ring, barriers and scratch.
__host__ __device__ inline size_t xu_smem(int J, int nst) {
    (void)J;
    return 1024 + (size_t)nst * XU_STAGE_BYTES + 512;
}
// Largest ring depth that fits the 227 KB per-CTA limit and is a multiple of
// the converter groups (0: none fits).
inline int xu_stages(int J) {
    const size_t cap = 232448;
    for (int nst = XU_MAX_STAGES; nst >= 2; --nst)
        if (nst % XU_CONV_GROUPS == 0 && xu_smem(J, nst) <= cap) return nst;
    return 0;
}

// Q_V (J×R FP32 row-major) into xu_slabs(J) swizzled slabs (see above).
static __global__ void k_qv_tf32(const float *__restrict__ QV, int J, int R, float *__restrict__ out) {
    const int nslab = xu_slabs(J);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;      // (slab, row, k)
    if (i >= nslab * 64 * 32) return;
    const int sl = i / 2048, n = (i / 32) % 64, kc = i % 32;
    const int j = 32 * sl + kc, r = n & 31;
    float v = 0.f;
    if (j < J && r < R) {
        const float q = QV[(int64_t)j * R + r];
        const float big = tf32_rn(q);
        v = n < 32 ? big : tf32_rn(q - big);
    }
    reinterpret_cast<float *>(reinterpret_cast<char *>(out) + (size_t)sl * XU_SLAB_BYTES + umma::swz(n, kc))[0] = v;
}

// Index self-check: record a failed check (count in err[4], the first code
// in err[5]) so that the host reports it; the caller skips the access.
__device__ __forceinline__ void tc05_check_failed(int *err, int code) {
    if (atomicAdd(err + 4, 1) == 0) err[5] = code;
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
    const int nslab = xu_slabs(a.J), nst = a.nst;
    const int nstg = nslab / 2;                       // stages per tile (64 columns each)
    uint8_t *sX = sm;                                 // stage s: X boxes, then its Q_V slabs
    uint64_t *full = reinterpret_cast<uint64_t *>(sX + (size_t)nst * XU_STAGE_BYTES);
    uint64_t *conv = full + nst, *empty = conv + nst;
    uint64_t *accf = empty + nst, *acce = accf + XU_NACC, *done = acce + XU_NACC;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
    double *red = reinterpret_cast<double *>(tslot + 2);      // one per converter warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = (a.N_gen + 127) / 128;
    const int my_nt = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int total = my_nt * nstg;
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
            int issued = 0;
            for (int it = 0; it < total; ++it) {
                const int s = it % nst, u = it / nst;
                const long long w0 = xu_clk(a.pc);
                if (u > 0 && !umma::wait_or_abort(&empty[s], (uint32_t)(u - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                c_wait += xu_clk(a.pc) - w0;
                const int64_t tile = blockIdx.x + (int64_t)(it / nstg) * gridDim.x;
                const int kk = it % nstg;
                uint8_t *st = sX + (size_t)s * XU_STAGE_BYTES;
                mbar_expect_tx(&full[s], XU_STAGE_BYTES);
                if (tile * 128 >= a.N_gen || 64 * kk >= a.J + 64 || 2 * kk + 1 >= nslab) {
                    tc05_check_failed(a.err, 101);
                } else if (!(a.skip_first_copy && blockIdx.x == 0 && it == 0)) {
                    umma::tma_load_2d(st, &tmX, 64 * kk, (int)(tile * 128), &full[s]);
                    umma::tma_load_2d(st + XU_BOX_BYTES, &tmX, 64 * kk + 32, (int)(tile * 128), &full[s]);
                    bulk_g2s(st + XU_XBYTES, a.qv_slabs + (size_t)(2 * kk) * (XU_SLAB_BYTES / 4),
                             2 * XU_SLAB_BYTES, &full[s]);
                }
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
            if (a.pc) atomicAdd(&a.pc[0], (unsigned long long)c_wait);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0 && total > 0) {
            constexpr uint32_t id64 = umma::idesc_tf32(128, 64, 0, 0);
            constexpr uint32_t id32 = umma::idesc_tf32(128, 32, 0, 0);
            const uint32_t sx0 = smem_u32(sX);
            for (int it = 0; it < total; ++it) {
                const int s = it % nst, u = it / nst;
                const int kk = it % nstg;
                const int ab = it % XU_NACC, v = it / XU_NACC;
                const long long w0 = xu_clk(a.pc);
                if (v > 0 && !umma::wait_or_abort(&acce[ab], (uint32_t)(v - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                if (!umma::wait_or_abort(&conv[s], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit)) break;
                c_wait += xu_clk(a.pc) - w0;
                umma::fence_after();
                const uint32_t acol = tmem + 256u + (uint32_t)s * 64u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t dcol = tmem + (uint32_t)ab * 128u + 64u * h;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t st0 = sx0 + (uint32_t)s * XU_STAGE_BYTES;
                        const uint64_t ad = umma::sdesc_sw128(st0 + (uint32_t)h * XU_BOX_BYTES + 32u * k, 16, 1024);
                        const uint64_t bd = umma::sdesc_sw128(
                            st0 + XU_XBYTES + (uint32_t)h * XU_SLAB_BYTES + 32u * k, 16, 1024);
                        umma::mma_ss(dcol, ad, bd, id64, k != 0);
                        umma::mma_ts(dcol + 32u, acol + 32u * h + 8u * k, bd, id32, 1u);
                    }
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
    } else if (warp < XU_EPI_W0) {
        // ---- converters: group gr takes stages it ≡ gr (mod XU_CONV_GROUPS);
        // thread = tile row r, TMEM lane r ----
        const int q = warp & 3, gr = (warp - XU_CONV_W0) >> 2, r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        double xn = 0.0;
        for (int it = gr; it < total; it += XU_CONV_GROUPS) {
            const int s = it % nst, u = it / nst;
            const long long w0 = xu_clk(a.pc);
            const bool ok = umma::wait_or_abort(&full[s], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) break;
            c_wait += xu_clk(a.pc) - w0;
            float xs = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint8_t *row = sX + (size_t)s * XU_STAGE_BYTES + (size_t)h * XU_BOX_BYTES + (size_t)r * 128;
                uint32_t sv[32];
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    const float4 x = *reinterpret_cast<const float4 *>(row + ((c4 ^ (r & 7)) << 4));
                    const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        xs = fmaf(xv[e], xv[e], xs);
                        sv[4 * c4 + e] = __float_as_uint(tf32_rn(xv[e] - tf32_trunc(xv[e])));
                    }
                }
                umma::tmem_st32(lane_base + 256u + (uint32_t)s * 64u + 32u * h, sv);
            }
            xn += (double)xs;
            umma::tmem_st_wait();
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&conv[s]);
        }
        xn = warp_sum(xn);
        if (lane == 0) red[warp - XU_CONV_W0] = xn;
        if (a.pc && lane == 0) atomicAdd(&a.pc[2], (unsigned long long)c_wait);
    } else {
        // ---- epilogue: group gr takes stages it ≡ gr (mod XU_EPI_GROUPS);
        // thread = tile row r.  With two groups every thread runs the same
        // hand-over barriers per tile, also after an abort (then without
        // waiting or touching tensor memory). ----
        const int q = warp & 3, gr = (warp - XU_EPI_W0) >> 2, r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        bool dead = false;
        for (int tc = 0; tc < my_nt; ++tc) {
            float acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
            for (int kk = 0; kk < nstg; ++kk) {
                const int it = tc * nstg + kk;
                if ((it % XU_EPI_GROUPS) != gr || dead) continue;
                const int ab = it % XU_NACC, v = it / XU_NACC;
                const long long w0 = xu_clk(a.pc);
                const bool ok = umma::wait_or_abort(&accf[ab], (uint32_t)v & 1u, abort_f, a.err, a.wait_limit);
                if (!__all_sync(0xffffffffu, ok)) {
                    dead = true;
                    continue;
                }
                c_wait += xu_clk(a.pc) - w0;
                umma::fence_after();
                // per box: main terms (columns 0-31), then corrections (32-63),
                // 16 columns at a time
#pragma unroll
                for (int q4 = 0; q4 < 8; ++q4) {
                    uint32_t t[16];
                    umma::tmem_ld16(lane_base + (uint32_t)ab * 128u + 16u * q4, t);
                    umma::tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[16 * (q4 & 1) + c] += __uint_as_float(t[c]);
                }
                umma::fence_before();
                __syncwarp();
                if (lane == 0) umma::mbar_arrive(&acce[ab]);
            }
            if (XU_EPI_GROUPS == 2) {
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
                }
            }
            if (gr == 0 && !dead) {
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
            if (XU_EPI_GROUPS == 2) {
                umma::fence_before();
                asm volatile("bar.sync 2, 256;" ::: "memory");
                umma::fence_after();
            }
        }
        if (a.pc && lane == 0) atomicAdd(&a.pc[3], (unsigned long long)c_wait);
    }
    umma::fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int q = 0; q < 4 * XU_CONV_GROUPS; ++q) sum += red[q];
        a.xn_part[blockIdx.x] = sum;
        if (a.pc) atomicAdd(&a.pc[4], (unsigned long long)(clock64() - c_start));
    }
    if (warp == 0) {
        umma::fence_after();
        umma::tmem_free(tmem, XU_TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// k_xq_umma_rq: the same P' = X·Q_V (and the same MMAs in the same order, so
// the same bits) with all of Q_V's slabs resident in shared memory, which
// lets a stage's X be released as soon as the converters have read it.  In
// k_xq_umma a stage holds its X until the MMAs that read big(X) from shared
// memory complete, so a ring slot is held for TMA latency + conversion +
// MMA + commit, and the ring turnover caps the pass near 4.7 TB/s.  Here the
// converters write both parts, big(X) (the TF32 truncation) and small(X), to
// one of two tensor-memory A buffers and release the X slot at once; the MMAs
// read A from tensor memory and B (Q_V) from the resident slabs.  Fits when
// the slabs and two X stages fit the 227 KB per-CTA limit (J <= 640).
//
// One persistent CTA per SM, 10 warps: 0 TMA producer (the Q_V slabs once,
// then two 128×32 X boxes per stage), 1 MMA issuer, 2-5 converters (thread =
// tile row r = TMEM lane r; one group takes every stage, so no converter can
// run ahead of another on a barrier; eight warps, one box each, measured
// 4 % slower), 6-9 epilogue (as in k_xq_umma).  Tensor memory:
// accumulators in columns 0-255 (two stages of two 64-column boxes), A
// buffers in 256-511 (per buffer and box: big in 32 columns, small in the
// next 32).  Barriers: full[s] (X landed), xfree[s] (X read), afull[b] /
// afree[b] (A buffer written / its MMAs done), accf / acce as in k_xq_umma.
constexpr int XR_THREADS = 320;
constexpr int XR_MAX_STAGES = 6;
__host__ __device__ inline size_t xr_smem(int J, int nst) {
    return 1024 + (size_t)xu_slabs(J) * XU_SLAB_BYTES + (size_t)nst * XU_XBYTES + 512;
}
// X ring depth of k_xq_umma_rq for J columns (0: the slabs and two stages do
// not fit).
inline int xr_stages(int J) {
    const size_t cap = 232448;
    for (int nst = XR_MAX_STAGES; nst >= 2; --nst)
        if (xr_smem(J, nst) <= cap) return nst;
    return 0;
}

static __global__ void __launch_bounds__(XR_THREADS, 1)
    k_xq_umma_rq(const __grid_constant__ CUtensorMap tmX, XuArgs a) {
    extern __shared__ uint8_t xr_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(xr_raw) + 1023) & ~(uintptr_t)1023);
    const int nslab = xu_slabs(a.J), nst = a.nst;
    const int nstg = nslab / 2;                        // stages per tile (64 columns each)
    uint8_t *sQ = sm;                                  // resident Q_V slabs
    uint8_t *sX = sQ + (size_t)nslab * XU_SLAB_BYTES;  // X ring: two boxes per stage
    uint64_t *full = reinterpret_cast<uint64_t *>(sX + (size_t)nst * XU_XBYTES);
    uint64_t *xfree = full + nst;
    uint64_t *afull = xfree + nst, *afree = afull + 2;
    uint64_t *accf = afree + 2, *acce = accf + XU_NACC, *qfull = acce + XU_NACC, *done = qfull + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
    double *red = reinterpret_cast<double *>(tslot + 2);      // one per converter warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = (a.N_gen + 127) / 128;
    const int my_nt = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int total = my_nt * nstg;
    const long long c_start = xu_clk(a.pc);
    long long c_wait = 0;
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < nst; ++s2) {
            mbar_init(&full[s2], 1);
            mbar_init(&xfree[s2], 4);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&afull[b], 4);
            mbar_init(&afree[b], 1);
        }
        for (int b = 0; b < XU_NACC; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(qfull, 1);
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
            int issued = 0;
            mbar_expect_tx(qfull, (uint32_t)nslab * XU_SLAB_BYTES);
            for (int q = 0; q < nslab; ++q)
                bulk_g2s(sQ + (size_t)q * XU_SLAB_BYTES, a.qv_slabs + (size_t)q * (XU_SLAB_BYTES / 4),
                         XU_SLAB_BYTES, qfull);
            for (int it = 0; it < total; ++it) {
                const int s2 = it % nst, u = it / nst;
                const long long w0 = xu_clk(a.pc);
                if (u > 0 && !umma::wait_or_abort(&xfree[s2], (uint32_t)(u - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                c_wait += xu_clk(a.pc) - w0;
                const int64_t tile = blockIdx.x + (int64_t)(it / nstg) * gridDim.x;
                const int kk = it % nstg;
                uint8_t *st = sX + (size_t)s2 * XU_XBYTES;
                mbar_expect_tx(&full[s2], XU_XBYTES);
                if (tile * 128 >= a.N_gen || 64 * kk >= a.J + 64) {
                    tc05_check_failed(a.err, 111);
                } else if (!(a.skip_first_copy && blockIdx.x == 0 && it == 0)) {
                    umma::tma_load_2d(st, &tmX, 64 * kk, (int)(tile * 128), &full[s2]);
                    umma::tma_load_2d(st + XU_BOX_BYTES, &tmX, 64 * kk + 32, (int)(tile * 128), &full[s2]);
                }
                ++issued;
            }
            // copies still in flight land before the CTA exits
            {
                const long long t0 = clock64();
                while (!mbar_try_wait(qfull, 0) && clock64() - t0 < a.wait_limit) {
                }
            }
            for (int it = issued - 1; it >= 0 && it >= issued - nst; --it) {
                const int s2 = it % nst, u = it / nst;
                const long long t0 = clock64();
                while (!mbar_try_wait(&full[s2], (uint32_t)u & 1u) && clock64() - t0 < a.wait_limit) {
                }
            }
            if (a.pc) atomicAdd(&a.pc[0], (unsigned long long)c_wait);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0 && total > 0) {
            constexpr uint32_t id64 = umma::idesc_tf32(128, 64, 0, 0);
            constexpr uint32_t id32 = umma::idesc_tf32(128, 32, 0, 0);
            const uint32_t sq0 = smem_u32(sQ);
            bool ok = umma::wait_or_abort(qfull, 0u, abort_f, a.err, a.wait_limit);
            for (int it = 0; ok && it < total; ++it) {
                const int b = it & 1, ub = it >> 1;
                const int kk = it % nstg;
                const int ab = it % XU_NACC, v = it / XU_NACC;
                const long long w0 = xu_clk(a.pc);
                if (v > 0 && !umma::wait_or_abort(&acce[ab], (uint32_t)(v - 1) & 1u, abort_f, a.err, a.wait_limit))
                    break;
                if (!umma::wait_or_abort(&afull[b], (uint32_t)ub & 1u, abort_f, a.err, a.wait_limit)) break;
                c_wait += xu_clk(a.pc) - w0;
                umma::fence_after();
                const uint32_t abuf = tmem + 256u + 128u * (uint32_t)b;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t dcol = tmem + (uint32_t)ab * 128u + 64u * h;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t bd = umma::sdesc_sw128(
                            sq0 + (uint32_t)(2 * kk + h) * XU_SLAB_BYTES + 32u * k, 16, 1024);
                        umma::mma_ts(dcol, abuf + 64u * h + 8u * k, bd, id64, k != 0);
                        umma::mma_ts(dcol + 32u, abuf + 64u * h + 32u + 8u * k, bd, id32, 1u);
                    }
                }
                umma::commit(&afree[b]);
                umma::commit(&accf[ab]);
            }
            // every MMA issued has completed before the tensor memory is freed
            umma::commit(done);
            const long long t0 = clock64();
            while (!mbar_try_wait(done, 0) && clock64() - t0 < a.wait_limit) {
            }
            if (a.pc) atomicAdd(&a.pc[1], (unsigned long long)c_wait);
        }
    } else if (warp < 6) {
        // ---- converters: every stage in order; thread = tile row r, TMEM lane r ----
        const int q = warp & 3, r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        double xn = 0.0;
        for (int it = 0; it < total; ++it) {
            const int s2 = it % nst, u = it / nst;
            const int b = it & 1, ub = it >> 1;
            const long long w0 = xu_clk(a.pc);
            bool ok = umma::wait_or_abort(&full[s2], (uint32_t)u & 1u, abort_f, a.err, a.wait_limit);
            if (ok && ub > 0) ok = umma::wait_or_abort(&afree[b], (uint32_t)(ub - 1) & 1u, abort_f, a.err, a.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) break;
            c_wait += xu_clk(a.pc) - w0;
            umma::fence_after();
            float xs = 0.f;
            uint32_t bg[2][32], sl[2][32];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint8_t *row = sX + (size_t)s2 * XU_XBYTES + (size_t)h * XU_BOX_BYTES + (size_t)r * 128;
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    const float4 x = *reinterpret_cast<const float4 *>(row + ((c4 ^ (r & 7)) << 4));
                    const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        xs = fmaf(xv[e], xv[e], xs);
                        const float big = tf32_trunc(xv[e]);
                        bg[h][4 * c4 + e] = __float_as_uint(big);
                        sl[h][4 * c4 + e] = __float_as_uint(tf32_rn(xv[e] - big));
                    }
                }
            }
            // the stage's X is in registers: its slot can be refilled
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&xfree[s2]);
            const uint32_t abuf = lane_base + 256u + 128u * (uint32_t)b;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                umma::tmem_st32(abuf + 64u * h, bg[h]);
                umma::tmem_st32(abuf + 64u * h + 32u, sl[h]);
            }
            xn += (double)xs;
            umma::tmem_st_wait();
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&afull[b]);
        }
        xn = warp_sum(xn);
        if (lane == 0) red[warp - 2] = xn;
        if (a.pc && lane == 0) atomicAdd(&a.pc[2], (unsigned long long)c_wait);
    } else {
        // ---- epilogue: thread = tile row r ----
        const int q = warp & 3, r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        bool dead = false;
        for (int tc = 0; tc < my_nt && !dead; ++tc) {
            float acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
            for (int kk = 0; kk < nstg; ++kk) {
                const int it = tc * nstg + kk;
                const int ab = it % XU_NACC, v = it / XU_NACC;
                const long long w0 = xu_clk(a.pc);
                const bool ok = umma::wait_or_abort(&accf[ab], (uint32_t)v & 1u, abort_f, a.err, a.wait_limit);
                if (!__all_sync(0xffffffffu, ok)) {
                    dead = true;
                    break;
                }
                c_wait += xu_clk(a.pc) - w0;
                umma::fence_after();
                // per box: main terms (columns 0-31), then corrections (32-63),
                // 16 columns at a time
#pragma unroll
                for (int q4 = 0; q4 < 8; ++q4) {
                    uint32_t t[16];
                    umma::tmem_ld16(lane_base + (uint32_t)ab * 128u + 16u * q4, t);
                    umma::tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[16 * (q4 & 1) + c] += __uint_as_float(t[c]);
                }
                umma::fence_before();
                __syncwarp();
                if (lane == 0) umma::mbar_arrive(&acce[ab]);
            }
            if (dead) break;
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
        if (a.pc && lane == 0) atomicAdd(&a.pc[3], (unsigned long long)c_wait);
    }
    umma::fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int q = 0; q < 4; ++q) sum += red[q];
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
// (rank columns as MMA N, rows as K) is built in each stage's shared memory
// by builder warps from U and w_k,new, split and swizzled.  Per 32-row
// block and k-step of 8 rows:
//   D[:, 0:64]  (+)= big(X)ᵀ · [big(Ũ) | small(Ũ)]     (M=128, N=64)
//   D[:, 32:64]  += small(X)ᵀ · big(Ũ)                   (M=128, N=32)
// Every stage accumulates into a fresh accumulator of a ring of FB_NACC in
// tensor memory (4 k-steps each), which the epilogue warps add to FP32
// register sums (main + correction added in FP32, rounded to nearest): the
// same split of the sum as the X·Q_V pass.
constexpr int FB_THREADS = 384;
constexpr int FB_ROWS = 64;                    // rows per stage
constexpr int FB_XSTAGE = FB_ROWS * 128 * 4;   // 64 rows × 128 columns of X
constexpr int FB_UBLK = 64 * 128;              // Ũ block: 64 rank rows × 32 rows
constexpr int FB_STAGE = FB_XSTAGE + 2 * FB_UBLK;
constexpr int FB_NST = 3;
constexpr int FB_NACC = 2;
constexpr int FB_FLUSH = 16;                   // stages summed in registers before the outer sum
constexpr int FB_TMEM_COLS = 512;              // accumulators 0-127, A slots from 128 (128 each)

__host__ __device__ inline size_t fb_smem() { return 1024 + (size_t)FB_NST * FB_STAGE + 512; }

struct FbArgs {
    BatchDev b;              // the batch: general row → batch row → slice
    const float *U;          // U_k,new rows (batch row order, R per row)
    const float *Wf;         // FP32 copy of the new weights w_k,new (K×R)
    int64_t n_part;          // partial slots available in Fpart
    float *Fpart;            // per row chunk: J×R FP32 partial
    int *err;
    int64_t N_gen;
    int64_t rows_per_cta;    // a multiple of FB_ROWS
    int J, R;
    long long wait_limit;
};

// CTA (c, t): rows [c·rows_per_cta, ...) of the general rows, columns
// [128t, 128t + 128).  Warps: 0 producer (TMA box of 64 rows × 128 columns,
// no swizzle), 1 MMA issuer, 2-5 converters (thread = column j = TMEM lane),
// 6-9 epilogue (thread = column j), 10-11 Ũ builders (warp 10 + h builds the
// stage's 32-row block h; thread = row).  full[s] completes on the X bytes
// and the two builders' arrivals.
//
// Ũ(g, r) = U(row(g), r)·w_k,new(r), the FP32 product with the FP32 copy of
// the new weights, split into big = TF32(Ũ) and small = TF32(Ũ − big) and
// stored per 32-row block at rank row r (big) and 32 + r (small), K position
// g mod 32, 128-byte swizzled; rows past N_gen and ranks past R are zero.  A
// builder loads its rows before it waits for the stage to be free, so the
// loads overlap the wait.
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
    const int nstage = g1 > g0 ? (int)((g1 - g0 + FB_ROWS - 1) / FB_ROWS) : 0;
    const int j0 = 128 * blockIdx.y;
    if (threadIdx.x == 0) {
        for (int s = 0; s < FB_NST; ++s) {
            mbar_init(&full[s], 3);
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
                if (g0 + FB_ROWS * i >= a.N_gen || j0 >= a.J) {
                    tc05_check_failed(a.err, 301);   // stage skipped: its waits run out
                    break;
                }
                mbar_expect_tx(&full[s], FB_XSTAGE);
                umma::tma_load_2d(st, &tmX, j0, (int)(g0 + FB_ROWS * i), &full[s]);
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
                const uint32_t abig = tmem + 128u + (uint32_t)s * 128u;
                const uint32_t ub = s0 + (uint32_t)s * FB_STAGE + FB_XSTAGE;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint64_t bd = umma::sdesc_sw128(ub + (uint32_t)(k >> 2) * FB_UBLK + 32u * (k & 3), 16, 1024);
                    umma::mma_ts(dcol, abig + 8u * k, bd, id64, k != 0);
                    umma::mma_ts(dcol + 32u, abig + 64u + 8u * k, bd, id32, 1u);
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
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t bg[32], sl[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const float x = xs[(32 * h + r) * 128];
                    const float big = tf32_rn(x);
                    bg[r] = __float_as_uint(big);
                    sl[r] = __float_as_uint(tf32_rn(x - big));
                }
                umma::tmem_st32(lane_base + 128u + (uint32_t)s * 128u + 32u * h, bg);
                umma::tmem_st32(lane_base + 128u + (uint32_t)s * 128u + 64u + 32u * h, sl);
            }
            umma::tmem_st_wait();
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&conv[s]);
        }
    } else if (warp < 10) {
        // ---- epilogue: thread = column jl ----
        const int q = warp & 3, jl = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        // two-level FP32 sum: FB_FLUSH stages in acc, then into tot, so that
        // no running sum takes more than a few dozen terms
        float acc[32], tot[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = tot[r] = 0.f;
        bool ok_all = true;
        for (int i = 0; i < nstage; ++i) {
            const int ab = i % FB_NACC, v = i / FB_NACC;
            const bool ok = umma::wait_or_abort(&accf[ab], (uint32_t)v & 1u, abort_f, a.err, a.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) {
                ok_all = false;
                break;
            }
            umma::fence_after();
            // 16 rank columns at a time (main and correction), which keeps the
            // register count within the 448-thread block's share
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                uint32_t mn[16], cr[16];
                umma::tmem_ld16(lane_base + (uint32_t)ab * 64u + (uint32_t)c0, mn);
                umma::tmem_ld16(lane_base + (uint32_t)ab * 64u + 32u + (uint32_t)c0, cr);
                umma::tmem_ld_wait();
#pragma unroll
                for (int r = 0; r < 16; ++r) acc[c0 + r] += __uint_as_float(mn[r]) + __uint_as_float(cr[r]);
            }
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&acce[ab]);
            if ((i + 1) % FB_FLUSH == 0) {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    tot[r] += acc[r];
                    acc[r] = 0.f;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) tot[r] += acc[r];
        const int j = j0 + jl;
        if (ok_all && j < a.J && blockIdx.x >= a.n_part) {
            tc05_check_failed(a.err, 302);
        } else if (ok_all && j < a.J) {
            float *out = a.Fpart + (int64_t)blockIdx.x * a.J * a.R + (int64_t)j * a.R;
#pragma unroll
            for (int r = 0; r < 32; ++r)
                if (r < a.R) out[r] = tot[r];
        }
    } else {
        // ---- Ũ builders: warp 10 + h, thread = row 32h + lane of a stage.
        // Software-pipelined so that no global load sits on the critical
        // path: the batch row and slice of stage i + 2 and the U and w_new
        // rows of stage i + 1 are fetched while stage i is stored. ----
        const int h = warp - 10;
        const int64_t run0 = run0_of(a.b);
        const bool vec = (a.R & 3) == 0;
        auto locate = [&](int i, int64_t &row, int &k) {
            const int64_t g = g0 + (int64_t)FB_ROWS * i + 32 * h + lane;
            row = -1;
            k = 0;
            if (i < nstage && g < a.N_gen) {
                row = gen_row_fast(a.b, run0, g);
                k = __ldcg(a.b.row_slice + row);
            }
        };
        float x[32], wv[32];
        auto fetch = [&](int64_t row, int k) {
#pragma unroll
            for (int r = 0; r < 32; ++r) x[r] = wv[r] = 0.f;
            if (row < 0) return;
            const float *ur = a.U + row * a.R;
            const float *wr = a.Wf + (int64_t)k * a.R;
            if (vec) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (4 * q < a.R) {
                        const float4 u4 = __ldcg(reinterpret_cast<const float4 *>(ur) + q);
                        const float4 w4 = __ldcg(reinterpret_cast<const float4 *>(wr) + q);
                        x[4 * q] = u4.x; x[4 * q + 1] = u4.y; x[4 * q + 2] = u4.z; x[4 * q + 3] = u4.w;
                        wv[4 * q] = w4.x; wv[4 * q + 1] = w4.y; wv[4 * q + 2] = w4.z; wv[4 * q + 3] = w4.w;
                    }
            } else {
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    if (r < a.R) {
                        x[r] = __ldcg(ur + r);
                        wv[r] = __ldcg(wr + r);
                    }
            }
        };
        int64_t row_a, row_b;
        int k_a, k_b;
        locate(0, row_a, k_a);
        fetch(row_a, k_a);
        locate(1, row_b, k_b);
        for (int i = 0; i < nstage; ++i) {
            const int s = i % FB_NST, u = i / FB_NST;
            float v[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = x[r] * wv[r];
            fetch(row_b, k_b);                  // stage i + 1
            locate(i + 2, row_b, k_b);
            if (u > 0) {
                const bool ok = umma::wait_or_abort(&empty[s], (uint32_t)(u - 1) & 1u, abort_f, a.err, a.wait_limit);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            uint8_t *blk = sm + (size_t)s * FB_STAGE + FB_XSTAGE + (size_t)h * FB_UBLK;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const float big = tf32_rn(v[r]);
                *reinterpret_cast<float *>(blk + umma::swz(r, lane)) = big;
                *reinterpret_cast<float *>(blk + umma::swz(32 + r, lane)) = tf32_rn(v[r] - big);
            }
            // the MMAs read these stores through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&full[s]);
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
