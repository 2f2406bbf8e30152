// Mode-P (Algorithm 1) kernels, SIMT form, templated on the arithmetic type T
// of the bulk products (double or float) and the element type TI of X.
//
// One update runs, in stream order:
//   k_rowmap      row -> slice id of the staged batch                (P0)
//   k_xv          P = X_new V, plus ||X_new||² partials               (P3, Theorem 1)
//   k_slices      per slice: U_new = P M_k, c_k, D_k, W(k,:), G part   (P2, P4, P6, P7)
//   k_f           per-block partials of Σ_k X_k,newᵀ U_k,new S_k       (P5, Eq. 20)
//   k_f_reduce    F ← λF + Σ partials (fixed order)                   (P8, Eq. 20)
//   k_g_reduce    G ← λG + Σ partials (fixed order)                   (P8, Eq. 21)
//   k_pinv_small  G⁺                                                  (Eq. 17)
//   k_vupdate     V = F G⁺, cross term of the fitness                 (P9, Eq. 17)
//   k_gamma       Γ = VᵀV for the next update                         (P1)
//   k_gamma_inv   Γ⁺ and the batch fitness                            (P10)
// All reductions run in a fixed order (no floating-point atomics), so a
// batch gives bit-identical results however the launches interleave.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "small_linalg.cuh"

namespace dash {

// Per-slice summaries c_k, D_k are stored as FP64 (FP64 path) or as
// double-float pairs (mixed path); both are 8 bytes per entry.
template <bool DF> struct Summ;
template <> struct Summ<false> {
    static __device__ __forceinline__ double ld(const double *p, int64_t i) { return p[i]; }
    static __device__ __forceinline__ void st(double *p, int64_t i, double v) { p[i] = v; }
};
template <> struct Summ<true> {
    static __device__ __forceinline__ double ld(const double *p, int64_t i) {
        return df_to_double(reinterpret_cast<const df *>(p)[i]);
    }
    static __device__ __forceinline__ void st(double *p, int64_t i, double v) {
        reinterpret_cast<df *>(p)[i] = df_from_double(v);
    }
};

// Device view of one update's batch (built on the host from the staged
// segments).  Segment s covers rows seg_row[s]..seg_row[s+1]-1 of X.
struct BatchDev {
    int n_seg;
    int n_touch;            // slices with at least one segment
    int K_all;              // slices after this update (old + new)
    int K_old;              // slices before this update
    int64_t N;              // rows in the batch
    const int *seg_slice;   // [n_seg]
    const int64_t *seg_row; // [n_seg + 1]
    const int *tslot;       // [K_all] touched index of slice k, or -1
    const int *tseg_ptr;    // [n_touch + 1]
    const int *tseg_idx;    // segments of each touched slice, in batch order
    int *row_slice;         // [N] filled by k_rowmap
    // rows handled by the general kernels: n_runs runs of consecutive rows;
    // general row g lives at run_row0[r] + (g - run_g0[r]) for the run r
    // with run_g0[r] <= g < run_g0[r+1]
    int n_runs;
    int64_t N_gen;
    const int64_t *run_g0;  // [n_runs + 1]
    const int64_t *run_row0;// [n_runs]
};

__device__ __forceinline__ int64_t gen_row(const BatchDev &b, int64_t g) {
    int lo = 0, hi = b.n_runs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.run_g0[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return b.run_row0[lo] + (g - b.run_g0[lo]);
}

// Model state on the device (FP64 master copies).
struct StateDev {
    int J, R;
    double lam, rtol;
    double *V;        // J×R
    double *W;        // Kmax×R
    double *c;        // Kmax×R
    double *D;        // Kmax×R×R
    double *F;        // J×R
    double *G;        // R×R
    double *Gam;      // R×R  Γ = VᵀV
    double *GamP;     // R×R  Γ⁺
    int *gam_ok;      // Γ nonsingular (Cholesky path accepted)
};

template <typename T> __device__ __forceinline__ T to_t(double v) { return (T)v; }

// λ·x with λ = 0 meaning "drop the old term" (never 0·NaN)
__device__ __forceinline__ double lam_scale(double lam, double x) { return lam == 0.0 ? 0.0 : lam * x; }

// ---------------------------------------------------------------------------
// P0: new slices start with S_k = I (Lemma 1 for a slice without S_k), zero
// helpers.
static __global__ void k_begin_new(double *W, double *c, double *D, int K_old, int n_new, int R) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)n_new * R * (R + 2);
    if (i >= tot) return;
    const int64_t per = (int64_t)R * (R + 2);
    const int k = K_old + (int)(i / per);
    const int e = (int)(i % per);
    if (e < R) W[(int64_t)k * R + e] = 1.0;
    else if (e < 2 * R) c[(int64_t)k * R + (e - R)] = 0.0;
    else D[(int64_t)k * R * R + (e - 2 * R)] = 0.0;
}

static __global__ void k_rowmap(BatchDev b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    int lo = 0, hi = b.n_seg - 1;         // last segment with seg_row[s] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.seg_row[mid] <= i) lo = mid; else hi = mid - 1;
    }
    // skip empty segments that share the start row
    while (lo + 1 < b.n_seg && b.seg_row[lo + 1] <= i) ++lo;
    b.row_slice[i] = b.seg_slice[lo];
}

// ---------------------------------------------------------------------------
// P3: P = X_new V.  64 rows per CTA, 256 threads; thread t computes row t/4
// and columns t%4, t%4+4, ...  (R <= 64).  Also ||X||² partial per CTA.
constexpr int XV_ROWS = 64;
constexpr int XV_KC = 32;

template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_xv(const TI *__restrict__ X, BatchDev b, int J, int R,
                                            const T *__restrict__ VT, T *__restrict__ P,
                                            double *__restrict__ xn_part) {
    __shared__ T Xs[XV_ROWS][XV_KC + 1];
    __shared__ T Vs[XV_KC][kMaxR];
    __shared__ double red[8];
    __shared__ int64_t rows_s[XV_ROWS];
    const int tid = threadIdx.x;
    const int64_t N = b.N_gen;
    const int64_t row0 = (int64_t)blockIdx.x * XV_ROWS;   // general row index
    if (tid < XV_ROWS) rows_s[tid] = (row0 + tid < N) ? gen_row(b, row0 + tid) : -1;
    __syncthreads();
    const int ri = tid >> 2;
    const int cg = tid & 3;
    T acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = T(0);
    double xn = 0.0;
    for (int j0 = 0; j0 < J; j0 += XV_KC) {
        __syncthreads();
        for (int e = tid; e < XV_ROWS * XV_KC; e += 256) {
            const int r = e / XV_KC, jj = e % XV_KC;
            const int64_t row = rows_s[r];
            T v = T(0);
            if (row >= 0 && j0 + jj < J) {
                const TI x = X[row * J + j0 + jj];
                v = (T)x;
                xn += (double)x * (double)x;
            }
            Xs[r][jj] = v;
        }
        for (int e = tid; e < XV_KC * R; e += 256) {
            const int jj = e / R, r = e % R;
            Vs[jj][r] = (j0 + jj < J) ? VT[(int64_t)(j0 + jj) * R + r] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < XV_KC; ++jj) {
            const T x = Xs[ri][jj];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int r = cg + 4 * q;
                if (r < R) acc[q] += x * Vs[jj][r];
            }
        }
    }
    const int64_t row = rows_s[ri];
    if (row >= 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int r = cg + 4 * q;
            if (r < R) P[row * R + r] = acc[q];
        }
    }
    xn = warp_sum(xn);
    if ((tid & 31) == 0) red[tid >> 5] = xn;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        xn_part[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// P2, P4, P6, P7: one warp per slice, all K_all slices.
//   touched: M_k = S_k (S_k Γ S_k)⁺ (= Γ⁺ S_k⁻¹ when Γ and S_k are
//   nonsingular), U = P M_k written out, ΔD = UᵀU, Δc = Σ_i U∘P,
//   c ← λc + Δc, D ← λD + ΔD  (Eqs. 15, 16)
//   untouched: c ← λc, D ← λD
//   then W(k,:) = c_kᵀ (Γ ∗ D_k)⁺ (Eq. 12); the warp's share of
//   G_inc = Σ S_k ΔD_k S_k (Eq. 21) is reduced per CTA into Gpart.
__host__ __device__ inline int sl_ld(int R) { return R + 1; }
// doubles of shared memory per warp: M, A, E, DD, Gw (R×ld), Pc, Uc (32×ld),
// w, cv, f, dc (ld)
__host__ __device__ inline int sl_warp_doubles(int R) {
    const int ld = sl_ld(R);
    return 5 * R * ld + 64 * ld + 4 * ld;
}
// warps per CTA so that the CTA fits in 220 KB of shared memory
__host__ inline int sl_warps(int R) {
    const int per = sl_warp_doubles(R) * 8;
    int nw = (220 * 1024) / per;
    return nw < 1 ? 1 : (nw > 4 ? 4 : nw);
}

template <typename T, bool DF>
__global__ void __launch_bounds__(128) k_slices(BatchDev b, StateDev s,
                                               const T *__restrict__ P,
                                               T *__restrict__ U,
                                               double *__restrict__ Gpart) {
    extern __shared__ double sm[];
    const int R = s.R, ld = sl_ld(R);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    double *base = sm + (size_t)wid * sl_warp_doubles(R);
    double *M = base;                // R×ld  (also Cholesky workspace in the W solve)
    double *A = M + R * ld;          // R×ld
    double *E = A + R * ld;          // R×ld
    double *DD = E + R * ld;         // R×ld
    double *Gw = DD + R * ld;        // R×ld  (warp's G partial)
    double *Pc = Gw + R * ld;        // 32×ld
    double *Uc = Pc + 32 * ld;       // 32×ld
    double *w = Uc + 32 * ld;        // ld
    double *cv = w + ld;             // ld
    double *f = cv + ld;             // ld
    double *dc = f + ld;             // ld

    for (int i = lane; i < R * ld; i += 32) Gw[i] = 0.0;
    const int total_warps = gridDim.x * nw;
    for (int k = blockIdx.x * nw + wid; k < b.K_all; k += total_warps) {
        __syncwarp();
        const int t = b.tslot[k];
        if (t == -2) continue;                 // finished by the fused row kernel
        const double *Wk = s.W + (int64_t)k * R;
        double *ck = s.c + (int64_t)k * R;
        double *Dk = s.D + (int64_t)k * R * R;
        for (int i = lane; i < R * ld; i += 32) DD[i] = 0.0;
        for (int i = lane; i < R; i += 32) { w[i] = Wk[i]; dc[i] = 0.0; }
        __syncwarp();
        if (t >= 0) {
            // ---- M_k (Lemma 1) -------------------------------------------
            int nz = 0;
            for (int i = 0; i < R; ++i) nz += (w[i] != 0.0);
            if (nz == 0) {
                for (int i = lane; i < R * ld; i += 32) M[i] = 0.0;
            } else if (nz == R && *s.gam_ok) {
                for (int i = lane; i < R * R; i += 32) {
                    const int r = i / R, q = i % R;
                    M[r * ld + q] = s.GamP[r * R + q] / w[q];
                }
            } else {
                for (int i = lane; i < R * R; i += 32) {
                    const int r = i / R, q = i % R;
                    A[r * ld + q] = w[r] * s.Gam[r * R + q] * w[q];
                }
                __syncwarp();
                warp_psd_pinv(A, E, f, M, R, ld, s.rtol, 1, false);
                for (int i = lane; i < R * R; i += 32) {
                    const int r = i / R, q = i % R;
                    M[r * ld + q] *= w[r];
                }
            }
            __syncwarp();
            // ---- rows of every segment of slice k --------------------------
            for (int si = b.tseg_ptr[t]; si < b.tseg_ptr[t + 1]; ++si) {
                const int sg = b.tseg_idx[si];
                const int64_t r0 = b.seg_row[sg], r1 = b.seg_row[sg + 1];
                for (int64_t c0 = r0; c0 < r1; c0 += 32) {
                    const int nr = (int)(r1 - c0 < 32 ? r1 - c0 : 32);
                    __syncwarp();
                    for (int e = lane; e < nr * R; e += 32) {
                        const int i = e / R, r = e % R;
                        Pc[i * ld + r] = (double)P[(c0 + i) * R + r];
                    }
                    __syncwarp();
                    if (lane < nr) {
                        for (int q = 0; q < R; ++q) {
                            double u = 0.0;
                            for (int r = 0; r < R; ++r) u += Pc[lane * ld + r] * M[r * ld + q];
                            Uc[lane * ld + q] = u;
                        }
                    }
                    __syncwarp();
                    for (int e = lane; e < nr * R; e += 32) {
                        const int i = e / R, r = e % R;
                        U[(c0 + i) * R + r] = to_t<T>(Uc[i * ld + r]);
                    }
                    // ΔD (upper triangle) and Δc, one entry per lane
                    const int ne = R * (R + 1) / 2;
                    for (int e = lane; e < ne + R; e += 32) {
                        if (e < ne) {
                            int r = 0, rem = e;
                            while (rem >= R - r) { rem -= R - r; ++r; }
                            const int q = r + rem;
                            double a = 0.0;
                            for (int i = 0; i < nr; ++i) a += Uc[i * ld + r] * Uc[i * ld + q];
                            DD[r * ld + q] += a;
                        } else {
                            const int r = e - ne;
                            double a = 0.0;
                            for (int i = 0; i < nr; ++i) a += Uc[i * ld + r] * Pc[i * ld + r];
                            dc[r] += a;
                        }
                    }
                }
            }
            __syncwarp();
            for (int i = lane; i < R * R; i += 32) {       // mirror upper → lower
                const int r = i / R, q = i % R;
                if (r > q) DD[r * ld + q] = DD[q * ld + r];
            }
            __syncwarp();
        }
        // ---- c_k, D_k with λ (Eqs. 15, 16), written back -------------------
        for (int i = lane; i < R; i += 32) {
            const double v = lam_scale(s.lam, Summ<DF>::ld(ck, i)) + dc[i];
            cv[i] = v;
            Summ<DF>::st(ck, i, v);
        }
        for (int i = lane; i < R * R; i += 32) {
            const int r = i / R, q = i % R;
            const double v = lam_scale(s.lam, Summ<DF>::ld(Dk, i)) + DD[r * ld + q];
            Summ<DF>::st(Dk, i, v);
            A[r * ld + q] = s.Gam[i] * v;               // Γ ∗ D_k
        }
        __syncwarp();
        // ---- W(k,:) = c_kᵀ (Γ ∗ D_k)⁺ (Eq. 12) --------------------------------
        warp_psd_solve(A, M, E, cv, f, R, ld, s.rtol);
        double *Wout = s.W + (int64_t)k * R;
        for (int i = lane; i < R; i += 32) Wout[i] = cv[i];
        __syncwarp();
        // ---- G_inc share: S_k ΔD_k S_k with the new S_k (Eq. 21) -----------
        if (t >= 0) {
            for (int i = lane; i < R * R; i += 32) {
                const int r = i / R, q = i % R;
                Gw[r * ld + q] += cv[r] * DD[r * ld + q] * cv[q];
            }
        }
    }
    __syncthreads();
    // fixed-order reduction of the warps' G partials
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        const int r = i / R, q = i % R;
        double a = 0.0;
        for (int wv = 0; wv < nw; ++wv) {
            const double *g = sm + (size_t)wv * sl_warp_doubles(R) + 4 * R * ld;
            a += g[r * ld + q];
        }
        Gpart[(int64_t)blockIdx.x * R * R + i] = a;
    }
}

// ---------------------------------------------------------------------------
// P5: partials of F_inc = Σ_k X_k,newᵀ U_k,new S_k,new (Eq. 20).  CTA
// (bx, by) covers rows of chunk bx and columns j in [64·by, 64·by+64);
// thread t accumulates j = t%64, r = t/64 + 4q.
constexpr int F_JB = 64;
constexpr int F_RC = 32;

template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_f(const TI *__restrict__ X, BatchDev b, int J, int R,
                                           const T *__restrict__ U, const double *__restrict__ W,
                                           int64_t rows_per_chunk, T *__restrict__ Fpart) {
    __shared__ T Xs[F_RC][F_JB + 1];
    __shared__ T Us[F_RC][kMaxR];
    __shared__ int64_t rows_s[F_RC];
    const int tid = threadIdx.x;
    const int jj = tid % F_JB, rg = tid / F_JB;
    const int j0 = blockIdx.y * F_JB;
    const int64_t rbeg = (int64_t)blockIdx.x * rows_per_chunk;     // general row indices
    const int64_t rend = (b.N_gen < rbeg + rows_per_chunk) ? b.N_gen : rbeg + rows_per_chunk;
    T acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = T(0);
    for (int64_t c0 = rbeg; c0 < rend; c0 += F_RC) {
        const int nr = (int)(rend - c0 < F_RC ? rend - c0 : F_RC);
        __syncthreads();
        if (tid < F_RC) rows_s[tid] = tid < nr ? gen_row(b, c0 + tid) : 0;
        __syncthreads();
        for (int e = tid; e < F_RC * F_JB; e += 256) {
            const int i = e / F_JB, j = e % F_JB;
            Xs[i][j] = (i < nr && j0 + j < J) ? (T)X[rows_s[i] * J + j0 + j] : T(0);
        }
        for (int e = tid; e < F_RC * R; e += 256) {
            const int i = e / R, r = e % R;
            T v = T(0);
            if (i < nr) {
                const int64_t row = rows_s[i];
                const int k = b.row_slice[row];
                v = U[row * R + r] * (T)W[(int64_t)k * R + r];
            }
            Us[i][r] = v;
        }
        __syncthreads();
        for (int i = 0; i < nr; ++i) {
            const T x = Xs[i][jj];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int r = rg + 4 * q;
                if (r < R) acc[q] += x * Us[i][r];
            }
        }
    }
    if (j0 + jj < J) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int r = rg + 4 * q;
            if (r < R) Fpart[((int64_t)blockIdx.x * J + j0 + jj) * R + r] = acc[q];
        }
    }
}

// The kernels below that write the model's state take `abandoned` (may be
// null): when *abandoned != 0 a bounded wait of this update timed out, the
// update is dropped and they leave the state as it was.

// P8: F ← λF + Σ_b Fpart[b] (Eq. 20); F_inc kept for the fitness.
template <typename T>
__global__ void k_f_reduce(const T *__restrict__ Fpart, int nb, int J, int R, double lam,
                           double *__restrict__ F, double *__restrict__ Finc,
                           const int *__restrict__ abandoned) {
    if (abandoned && *abandoned) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)J * R) return;
    double a = 0.0;
    for (int p = 0; p < nb; ++p) a += (double)Fpart[(int64_t)p * J * R + i];
    Finc[i] = a;
    F[i] = lam_scale(lam, F[i]) + a;
}

// P8: G ← λG + Σ partials (Eq. 21), one warp per entry, fixed lane order.
static __global__ void k_g_reduce(const double *__restrict__ Gpart, int nb, int R, double lam,
                           double *__restrict__ G, double *__restrict__ Ginc,
                           const int *__restrict__ abandoned) {
    if (abandoned && *abandoned) return;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= R * R) return;
    double a = 0.0;
    for (int p = lane; p < nb; p += 32) a += Gpart[(int64_t)p * R * R + e];
    a = warp_sum(a);
    if (lane == 0) {
        Ginc[e] = a;
        G[e] = lam_scale(lam, G[e]) + a;
    }
}

// G⁺ (or Γ⁺) of a symmetric PSD R×R matrix by one warp; ok (optional)
// receives 1 when the Cholesky path was taken.
static __global__ void k_pinv_small(const double *__restrict__ Min, int R, double rtol,
                             double *__restrict__ Mout, int *ok, const int *__restrict__ abandoned) {
    if (abandoned && *abandoned) return;
    extern __shared__ double sm[];
    const int ld = R + 1, lane = threadIdx.x & 31;
    double *A = sm, *E = A + R * ld, *out = E + R * ld, *f = out + R * ld;
    for (int i = lane; i < R * R; i += 32) A[(i / R) * ld + (i % R)] = Min[i];
    __syncwarp();
    // Cholesky acceptance is decided inside warp_psd_pinv; detect it by
    // re-running the pivot test here for the flag.
    double md = 0.0;
    for (int i = lane; i < R; i += 32) md = fmax(md, fabs(A[i * ld + i]));
    md = warp_max(md);
    for (int i = lane; i < R * R; i += 32) E[(i / R) * ld + (i % R)] = A[(i / R) * ld + (i % R)];
    __syncwarp();
    const bool chol = md > 0.0 && warp_cholesky(E, R, ld, 100.0 * rtol * md);
    __syncwarp();
    warp_psd_pinv(A, E, f, out, R, ld, rtol, 1, chol);
    for (int i = lane; i < R * R; i += 32) Mout[i] = out[(i / R) * ld + (i % R)];
    if (ok && lane == 0) *ok = chol ? 1 : 0;
}

// G⁺ (or Γ⁺) of a symmetric PSD R×R matrix, R <= 32, spread over R CTAs of
// one warp (each on its own SM: the FP64 pipe is per SM).  Every CTA factors
// A = L Lᵀ in registers (lane l = row l, right-looking, pivots broadcast by
// shuffles); when every pivot exceeds 100·rtol·max(diag), CTA c writes
// column c of A⁻¹ by two triangular solves (forward from registers,
// backward from L in shared memory).  Otherwise CTA 0 alone takes the eigen
// path of k_pinv_small for the whole matrix.  ok (optional) receives 1 for
// the Cholesky path.  Dynamic shared memory: as k_pinv_small.
static __global__ void __launch_bounds__(32) k_pinv_cols(const double *__restrict__ Min, int R,
                                                         double rtol, double *__restrict__ Mout,
                                                         int *ok, const int *__restrict__ abandoned) {
    if (abandoned && *abandoned) return;
    extern __shared__ double sm[];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, ld = R + 1;
    const bool act = lane < R;
    double row[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) row[q] = (act && q < R) ? Min[lane * R + q] : 0.0;
    double md = 0.0;
#pragma unroll
    for (int q = 0; q < 32; ++q)
        if (q == lane) md = fabs(row[q]);
    md = warp_max(md);
    const double tol = 100.0 * rtol * md;
    bool chol = md > 0.0;
    double myinv = 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j < R) {
            const double piv = __shfl_sync(full, row[j], j);
            chol = chol && (piv > tol);
            const double inv = 1.0 / sqrt(piv > 0.0 ? piv : 1.0);
            const double lij = (lane == j) ? piv * inv : row[j] * inv;
            row[j] = lij;
            if (lane == j) myinv = inv;
#pragma unroll
            for (int q = j + 1; q < 32; ++q) {
                const double lqj = __shfl_sync(full, lij, q);
                if (q < R) row[q] = fma(-lij, lqj, row[q]);
            }
        }
    }
    if (chol) {
        double *Ls = sm;                       // L, row l at Ls[l·ld]
#pragma unroll
        for (int q = 0; q < 32; ++q)
            if (act && q < R && q <= lane) Ls[lane * ld + q] = row[q];
        __syncwarp();
        const int c = blockIdx.x;
        double y = (lane == c) ? 1.0 : 0.0;    // L y = e_c
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j < R) {
                const double yj = __shfl_sync(full, y * myinv, j);
                if (lane == j) y = yj;
                else if (lane > j && act) y = fma(-row[j], yj, y);
            }
        }
        for (int j = R - 1; j >= 0; --j) {     // Lᵀ x = y
            const double xj = __shfl_sync(full, y * myinv, j);
            if (lane == j) y = xj;
            else if (lane < j) y = fma(-Ls[j * ld + lane], xj, y);
        }
        if (act) Mout[lane * R + c] = y;
        if (ok && c == 0 && lane == 0) *ok = 1;
        return;
    }
    if (blockIdx.x != 0) return;
    double *A = sm, *E = A + R * ld, *out = E + R * ld, *f = out + R * ld;
    for (int i = lane; i < R * R; i += 32) A[(i / R) * ld + (i % R)] = Min[i];
    __syncwarp();
    warp_psd_pinv(A, E, f, out, R, ld, rtol, 1, false);
    for (int i = lane; i < R * R; i += 32) Mout[i] = out[(i / R) * ld + (i % R)];
    if (ok && lane == 0) *ok = 0;
}

// P9: V = F G⁺ (Eq. 17), one row per warp, plus V in T for the kernels and
// the fitness cross term Σ V ∗ F_inc per CTA.
template <typename T>
__global__ void k_vupdate(const double *__restrict__ F, const double *__restrict__ GP,
                          const double *__restrict__ Finc, int J, int R, double *__restrict__ V,
                          T *__restrict__ VT, double *__restrict__ cross_part,
                          const int *__restrict__ abandoned, int *nonfinite) {
    if (abandoned && *abandoned) return;
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int j = blockIdx.x * 8 + wid;
    double cr = 0.0;
    if (j < J) {
        for (int q = lane; q < R; q += 32) {
            double v = 0.0;
            for (int r = 0; r < R; ++r) v += F[(int64_t)j * R + r] * GP[r * R + q];
            V[(int64_t)j * R + q] = v;
            VT[(int64_t)j * R + q] = (T)v;
            if (nonfinite && !isfinite(v)) atomicAdd(nonfinite, 1);   // reported as DASH_ENUMERIC
            if (Finc) cr += v * Finc[(int64_t)j * R + q];
        }
    }
    cr = warp_sum(cr);
    if (lane == 0) red[wid] = cr;
    __syncthreads();
    if (threadIdx.x == 0 && cross_part) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        cross_part[blockIdx.x] = s;
    }
}

// P1: Γ = VᵀV, one warp per entry (r, q), lanes over j.
static __global__ void k_gamma(const double *__restrict__ V, int J, int R, double *__restrict__ Gam,
                               const int *__restrict__ abandoned) {
    if (abandoned && *abandoned) return;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= R * R) return;
    const int r = e / R, q = e % R;
    double a = 0.0;
    for (int j = lane; j < J; j += 32) a += V[(int64_t)j * R + r] * V[(int64_t)j * R + q];
    a = warp_sum(a);
    if (lane == 0) Gam[e] = a;
}

// V (FP64) → VT (T).
template <typename T>
__global__ void k_cast(const double *__restrict__ in, T *__restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}

// P10: batch fitness from FP64 Gram terms, one warp:
//   ||X − X̂||² = ||X||² − 2 Σ V ∗ F_inc + Σ Γ ∗ G_inc.
static __global__ void k_fitness(const double *__restrict__ xn_part, int n_xn,
                          const double *__restrict__ cross_part, int n_cross,
                          const double *__restrict__ Gam, const double *__restrict__ Ginc,
                          int R, const int *__restrict__ gam_ok,
                          double *__restrict__ out /* [fit, xnorm2, resid2, gam_ok] */) {
    const int lane = threadIdx.x & 31;
    double xn = 0.0, cr = 0.0, qd = 0.0;
    for (int i = lane; i < n_xn; i += 32) xn += xn_part[i];
    for (int i = lane; i < n_cross; i += 32) cr += cross_part[i];
    for (int i = lane; i < R * R; i += 32) qd += Gam[i] * Ginc[i];
    xn = warp_sum(xn);
    cr = warp_sum(cr);
    qd = warp_sum(qd);
    if (lane == 0) {
        const double res = fmax(0.0, xn - 2.0 * cr + qd);
        out[0] = xn > 0.0 ? 1.0 - sqrt(res / xn) : 1.0;
        out[1] = xn;
        out[2] = res;
        out[3] = (double)*gam_ok;
    }
}

// λ-weighted fitness of every row absorbed so far, each with the U_k,new
// S_k,new its update produced (the frozen products that enter F and G,
// Eqs. 20-21) and the current V: the residual Σ λ^age ||x − (u∘w)Vᵀ||² is
// xx − 2 tr(VᵀF) + tr(VᵀV G), xx = Σ λ^age ||x||².  One warp.
static __global__ void k_fit_lambda(const double *__restrict__ V, const double *__restrict__ F,
                                    const double *__restrict__ Gam, const double *__restrict__ G,
                                    int J, int R, double xx, double *__restrict__ out /* [fit, resid2] */) {
    const int lane = threadIdx.x & 31;
    double a = 0.0, q = 0.0;
    for (int i = lane; i < J * R; i += 32) a += V[i] * F[i];
    for (int i = lane; i < R * R; i += 32) q += Gam[i] * G[i];
    a = warp_sum(a);
    q = warp_sum(q);
    if (lane == 0) {
        const double res = fmax(0.0, xx - 2.0 * a + q);
        out[0] = xx > 0.0 ? 1.0 - sqrt(res / xx) : 1.0;
        out[1] = res;
    }
}

// Eq. 6 after the static fit: c_k = vec(X_k)ᵀ(V ⊙ U_k) = Σ_i U(i,:) ∘ P(i,:)
// with P = X V for the final V; one warp per touched slice, lanes over r.
template <typename T, bool DF>
__global__ void k_c_recompute(BatchDev b, const T *__restrict__ P, const T *__restrict__ U, int R,
                              double *__restrict__ c) {
    const int lane = threadIdx.x & 31;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwt = gridDim.x * (blockDim.x >> 5);
    for (int k = wg; k < b.K_all; k += nwt) {
        const int t = b.tslot[k];
        for (int r = lane; r < R; r += 32) {
            double a = 0.0;
            if (t >= 0) {
                for (int si = b.tseg_ptr[t]; si < b.tseg_ptr[t + 1]; ++si) {
                    const int sg = b.tseg_idx[si];
                    for (int64_t i = b.seg_row[sg]; i < b.seg_row[sg + 1]; ++i)
                        a += (double)U[i * R + r] * (double)P[i * R + r];
                }
            }
            Summ<DF>::st(c, (int64_t)k * R + r, a);
        }
    }
}

}  // namespace dash
