// Constrained-mode (U_k = Q_k H S_k) streaming update: the old/new split of
// Dash applied to PARAFAC2 with column-orthonormal Q_k.  Per update, in
// stream order:
//
//   k_xv          P = X_new V                                   (shared with mode P)
//   k_q_arows     A_new = P S_k Hᵀ, row by row
//   k_q_lt        per slice: L_k ← R factor of [√λ L_k; A_new]  (L_kᵀL_k = B_k),
//                 the eigenbasis of B_k, T_k = B_k^{-1/2} and B_k^{1/2},
//                 the carry matrix C_k = T_k,new·B_k,old^{1/2}, and the new
//                 rows of Q_k = A_new T_k
//   k_q_y         Y_k ← λ·C_k·Y_k + Q_k,newᵀX_new for every slice, with the
//                 per-CTA partials of the H-MTTKRP Σ_k Y_k V S_k and of WᵀW
//   k_q_h         H = (Σ_k Y_k V S_k)(VᵀV ∗ WᵀW)⁺ and (HᵀH ∗ WᵀW)⁺
//   k_q_vpart     V-MTTKRP shares Y_kᵀ H S_k
//   k_q_v         V = (Σ_k Y_kᵀ H S_k)(HᵀH ∗ WᵀW)⁺
//   k_gamma       VᵀV of the new V
//   k_q_pw        (HᵀH ∗ VᵀV)⁺
//   k_q_w         W(k,:) = diag(Hᵀ Y_k V)ᵀ (HᵀH ∗ VᵀV)⁺
//   k_q_out       the batch residual ‖X_new − Q_new H S_k Vᵀ‖² with the
//                 updated factors
// One CP-ALS sweep H → V → W on {Y_k}; with one batch on an empty model the
// whole update is one PARAFAC2-ALS iteration (Procrustes step + sweep).
//
// State per slice: L_k (B_k's triangular factor), the projected data
// Y_k = T_k Z_k = Q_kᵀΛ_kX_k (R×J) with Z_k = Σ λ^age A_kᵀX_k, and, as
// derived data, the eigenbasis E_k and B_k^{1/2}.  Y_k is carried instead
// of Z_k: its rows have the size of the data, while T_k's entries reach
// cond(A_k) (up to 1e6 on planted U(0,1) factors), so any product T_k·Z_k
// formed in FP32 would lose that many digits to cancellation.  The carry
// follows from Z_new = λZ_old + A_newᵀX_new:
//   Y_new = T_new Z_new = λ (T_new B_old^{1/2}) Y_old + Q_newᵀX_new,
// and since B_new ⪰ λB_old, ‖T_new B_old^{1/2}‖ <= λ^{-1/2}: the carry is a
// bounded R×R map, safe to apply in the product type.
//
// Precision: the bulk products (P, A, Y, the MTTKRPs, the residual) run in
// the product type T; everything that touches L_k or T_k runs in the scalar
// type S (double, or double-float in the mixed path).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dash_kernels_p.cuh"
#include "rr_linalg.cuh"
#include "small_linalg.cuh"

namespace dash {

struct QDev {
    int J, R;
    double lam, rtol;
    double *V;      // J×R
    double *H;      // R×R
    double *W;      // Kmax×R
    double *L;      // Kmax×R×R, upper-triangular factor of B_k (S storage: double or df)
    double *E;      // Kmax×R×R, eigenbasis of B_k (S storage)
    double *Bh;     // Kmax×R×R, B_k^{1/2} (S storage)
    double *C;      // Kmax×R×R, carry T_k,new B_k,old^{1/2} of this update (FP64)
    double *Gam;    // R×R  VᵀV (current V)
    int *err;       // [2]: slices whose factor or eigenvalues came out non-finite
    unsigned long long *phase;   // optional [4]: k_q_lt cycles in QR, FP32 pass, passes, tail
};

__host__ __device__ inline int q_ld(int R) { return R + 1; }

// P0 for mode Q: new slices start with w = 1, empty summaries and the
// identity as eigenbasis estimate.
template <class S, typename T>
__global__ void k_q_begin_new(double *W, double *Lraw, double *Eraw, double *Bhraw, T *Y, int K_old,
                              int n_new, int R, int J) {
    const int64_t per = (int64_t)R * (1 + 3 * R + J);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_new * per) return;
    const int k = K_old + (int)(i / per);
    int64_t e = i % per;
    S *L = reinterpret_cast<S *>(Lraw);
    S *E = reinterpret_cast<S *>(Eraw);
    S *Bh = reinterpret_cast<S *>(Bhraw);
    const int64_t RR = (int64_t)R * R;
    if (e < R) { W[(int64_t)k * R + e] = 1.0; return; }
    e -= R;
    if (e < RR) { L[k * RR + e] = RT<S>::zero(); return; }
    e -= RR;
    if (e < RR) { E[k * RR + e] = (e / R == e % R) ? RT<S>::one() : RT<S>::zero(); return; }
    e -= RR;
    if (e < RR) { Bh[k * RR + e] = RT<S>::zero(); return; }
    e -= RR;
    Y[(int64_t)k * R * J + e] = T(0);
}

// Q1 for R <= 32: A_new = P S_k Hᵀ, one warp per row (grid-stride).  Lane s
// forms P(i, s)·w_k(s) in T, and lane r sums those products against H(r, :)
// (staged in shared memory in T, transposed, padded) through shuffles.
template <typename T>
__global__ void __launch_bounds__(256) k_q_arows_w(int64_t N, int R, const int *__restrict__ row_slice,
                                                   const T *__restrict__ P, const double *__restrict__ W,
                                                   const double *__restrict__ H, T *__restrict__ A) {
    __shared__ T Ht[32 * 33];                      // Ht[s·33 + r] = H(r, s)
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int s2 = e / 32, r = e % 32;
        Ht[s2 * 33 + r] = (r < R && s2 < R) ? (T)H[r * R + s2] : T(0);
    }
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int64_t step = (int64_t)gridDim.x * wpb;
    for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < N; i += step) {
        const int k = row_slice[i];
        const T ps = lane < R ? P[i * R + lane] * (T)W[(int64_t)k * R + lane] : T(0);
        T a = T(0);
#pragma unroll
        for (int s2 = 0; s2 < 32; ++s2) a += __shfl_sync(full, ps, s2) * Ht[s2 * 33 + lane];
        if (lane < R) A[i * R + lane] = a;
    }
}

// Q1 for R > 32: A_new = P S_k Hᵀ, one thread per entry.
template <typename T>
__global__ void k_q_arows(int64_t N, int R, const int *__restrict__ row_slice,
                          const T *__restrict__ P, const double *__restrict__ W,
                          const double *__restrict__ H, T *__restrict__ A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * R) return;
    const int64_t i = e / R;
    const int r = (int)(e % R);
    const int k = row_slice[i];
    T a = T(0);
    for (int s = 0; s < R; ++s) a += P[i * R + s] * (T)(W[(int64_t)k * R + s] * H[r * R + s]);
    A[e] = a;
}

// Q3: per slice, one warp.
//   mode 0 (update): L_k ← √λ L_k, then the A rows of slice k folded in (QR);
//     eigen-decomposition of B_k = L_kᵀL_k warm-started from E_k; T_k and
//     B_k^{1/2}; the carry C_k = T_k B_k,old^{1/2} (FP64, λ > 0 only); the new
//     Q rows A_new T_k (product type).
//   mode 1 (prepare): E_k and B_k^{1/2} from a loaded L_k (cold start).
template <class S>
__host__ __device__ inline size_t q_lt_warp_bytes(int R) {
    // R <= 32: L, E and one scratch block (G, the rotations, T_k); larger R
    // also needs M for the Gram-Jacobi
    const int ld = q_ld(R);
    return (size_t)(R <= 32 ? 3 : 4) * R * ld * sizeof(S) + (size_t)3 * R * sizeof(S);
}

template <class S, typename T>
__global__ void k_q_lt(BatchDev b, QDev q, const T *__restrict__ A, T *__restrict__ Qrows, int mode,
                       int passes, float jac_tol) {
    using O = RT<S>;
    extern __shared__ unsigned char qlt_raw[];
    const int R = q.R, ld = q_ld(R);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned char *base = qlt_raw + (size_t)wid * q_lt_warp_bytes<S>(R);
    S *Lw = reinterpret_cast<S *>(base);
    S *Ew = Lw + R * ld;
    S *Gw = Ew + R * ld;      // G, the rotations, then T_k
    // R > 32: M, then B_old^{1/2}, B_new^{1/2}, staged A rows.  R <= 32 has no
    // fourth block: after the eigen-decomposition L_k (already written out)
    // is dead and its block takes those roles.
    S *Mw = R <= 32 ? Lw : Gw + R * ld;
    S *mu = (R <= 32 ? Gw : Mw) + R * ld;
    S *finv = mu + R;
    S *fsq = finv + R;
    const int chunk = R < 32 ? R : 32;      // A rows per QR step (staged in Gw)
    const S sl = O::from_d(sqrt(q.lam));
    const int64_t RR = (int64_t)R * R;
    S *Lg = reinterpret_cast<S *>(q.L);
    S *Eg = reinterpret_cast<S *>(q.E);
    S *Bg = reinterpret_cast<S *>(q.Bh);
    long long pc[4] = {0, 0, 0, 0};
    for (int k = blockIdx.x * nw + wid; k < b.K_all; k += gridDim.x * nw) {
        // the CTA's warps that have a slice in this pass take each phase (QR,
        // FP32 sweeps, Newton–Schulz, working-type sweeps, tail) together: a
        // named barrier over exactly those warps between phases, so that the
        // SM's instruction cache holds one phase's unrolled code at a time.
        // Every such warp runs the same barriers (none is data-dependent),
        // and warps without a slice have left the loop.
        const int kb = k - wid;
        const int nact = b.K_all - kb < nw ? b.K_all - kb : nw;
        auto phase_bar = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(32 * nact) : "memory"); };
        long long c0k = q.phase ? clock64() : 0;
        const int t = mode == 0 ? b.tslot[k] : -1;
        __syncwarp();
        for (int i = lane; i < R * R; i += 32) {
            const S v = Lg[k * RR + i];
            Lw[(i / R) * ld + (i % R)] = mode == 1 ? v : (q.lam == 0.0 ? O::zero() : O::mul(sl, v));
            Ew[(i / R) * ld + (i % R)] = mode == 1 ? ((i / R == i % R) ? O::one() : O::zero())
                                                   : Eg[k * RR + i];
        }
        __syncwarp();
        if (t >= 0) {
            for (int si = b.tseg_ptr[t]; si < b.tseg_ptr[t + 1]; ++si) {
                const int sg = b.tseg_idx[si];
                const int64_t r0 = b.seg_row[sg], r1 = b.seg_row[sg + 1];
                for (int64_t c0 = r0; c0 < r1; c0 += chunk) {
                    const int m = (int)(r1 - c0 < chunk ? r1 - c0 : chunk);
                    for (int e = lane; e < m * R; e += 32)
                        Gw[(e / R) * ld + (e % R)] = O::from_d((double)A[(c0 + e / R) * R + (e % R)]);
                    __syncwarp();
                    warp_qr_append(Lw, ld, Gw, ld, m, R);
                }
            }
        }
        if (mode == 0)
            for (int i = lane; i < R * R; i += 32) Lg[k * RR + i] = Lw[(i / R) * ld + (i % R)];
        if (q.phase) { const long long c1 = clock64(); pc[0] += c1 - c0k; c0k = c1; }
        phase_bar();
        if (R <= 32) {
            // register-resident one-sided Jacobi: FP32 sweeps, E re-orthogonalised
            // to the working type, then sweeps in the working type
            if (!std::is_same<S, float>::value) {
                // stops after the sweep that started below sqrt(1e-6)/2: the
                // quadratic step takes it to FP32's noise level
                warp_eig_os<float, S>(Lw, Ew, nullptr, R, ld, 8, 1e-6f, 5e-4f);
                phase_bar();
                // double-float: one step (the FP32 sweeps leave EᵀE − I at a few
                // 1e-6; one step takes it to about 1e-11, below the sweeps' 1e-10
                // target); FP64: two
                warp_newton_schulz_reg<S>(Ew, Gw, R, ld, std::is_same<S, df>::value ? 1 : 2);
            }
            if (q.phase) { const long long c1 = clock64(); pc[1] += c1 - c0k; c0k = c1; }
            phase_bar();
            // working-type sweeps; the double-float ones stop after the sweep that
            // started below sqrt(tol)/2 (quadratic convergence)
            warp_eig_os<S, S>(Lw, Ew, mu, R, ld, passes, jac_tol,
                              std::is_same<S, df>::value ? 0.5f * sqrtf(jac_tol) : 0.f);
            if (q.phase) { const long long c1 = clock64(); pc[2] += c1 - c0k; c0k = c1; }
            phase_bar();
        } else {
            // FP32 pre-pass (float scratch in G and M), then the working-type passes
            float *f0 = reinterpret_cast<float *>(Gw);
            const int fs = R * ld;
            if (!std::is_same<S, float>::value)
                warp_eig_prepass_f32<S>(Lw, Ew, f0, f0 + fs, f0 + 2 * fs, f0 + 3 * fs,
                                        reinterpret_cast<float *>(mu), Gw, Mw, R, ld, 6);
            if (q.phase) { const long long c1 = clock64(); pc[1] += c1 - c0k; c0k = c1; }
            phase_bar();
            warp_eig_factor(Lw, Ew, Gw, Mw, mu, R, ld, passes, jac_tol, 40, 1e-7f);
            if (q.phase) { const long long c1 = clock64(); pc[2] += c1 - c0k; c0k = c1; }
            phase_bar();
        }
        {
            // a non-finite factor or eigenvalue must not pass silently
            bool ok = true;
            for (int i = lane; i < R; i += 32) ok = ok && isfinite(O::to_d(mu[i]));
            for (int i = lane; i < R * R; i += 32) ok = ok && isfinite(O::to_d(Lw[(i / R) * ld + (i % R)]));
            if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicAdd(q.err + 2, 1);
        }
        warp_sqrt_weights(mu, R, q.rtol, finv, fsq);
        for (int i = lane; i < R * R; i += 32) Eg[k * RR + i] = Ew[(i / R) * ld + (i % R)];
        // T_k → Gw
        warp_spectral_s(Ew, finv, R, ld, Gw);
        if (mode == 0 && q.lam != 0.0) {
            // C_k = T_k · B_old^{1/2}  (B_old^{1/2} → Mw)
            for (int i = lane; i < R * R; i += 32) Mw[(i / R) * ld + (i % R)] = Bg[k * RR + i];
            __syncwarp();
            for (int idx = lane; idx < R * R; idx += 32) {
                const int r = idx / R, c = idx % R;
                S a = O::zero();
                for (int p = 0; p < R; ++p) a = O::fma(a, Gw[r * ld + p], Mw[p * ld + c]);
                q.C[k * RR + idx] = O::to_d(a);
            }
            __syncwarp();
        }
        // B_k^{1/2} → Mw → global
        warp_spectral_s(Ew, fsq, R, ld, Mw);
        for (int i = lane; i < R * R; i += 32) Bg[k * RR + i] = Mw[(i / R) * ld + (i % R)];
        // new Q rows = A_new T_k (A rows staged through Mw)
        if (t >= 0) {
            for (int si = b.tseg_ptr[t]; si < b.tseg_ptr[t + 1]; ++si) {
                const int sg = b.tseg_idx[si];
                const int64_t r0 = b.seg_row[sg], r1 = b.seg_row[sg + 1];
                for (int64_t c0 = r0; c0 < r1; c0 += chunk) {
                    const int m = (int)(r1 - c0 < chunk ? r1 - c0 : chunk);
                    __syncwarp();
                    for (int e = lane; e < m * R; e += 32)
                        Mw[(e / R) * ld + (e % R)] = O::from_d((double)A[(c0 + e / R) * R + (e % R)]);
                    __syncwarp();
                    for (int e = lane; e < m * R; e += 32) {
                        const int i = e / R, c = e % R;
                        S a = O::zero();
                        for (int p = 0; p < R; ++p) a = O::fma(a, Mw[i * ld + p], Gw[p * ld + c]);
                        Qrows[(c0 + i) * R + c] = (T)O::to_d(a);
                    }
                }
            }
        }
        __syncwarp();
        if (q.phase) pc[3] += clock64() - c0k;
    }
    if (q.phase && lane == 0)
        for (int i = 0; i < 4; ++i) atomicAdd(q.phase + i, (unsigned long long)pc[i]);
}

// Q2: Y_k ← λ C_k Y_k + Q_k,newᵀ X_new for every slice (λ C_k Y_k alone for
// untouched ones), then YV_k = Y_k V (old V) folded into the per-CTA
// H-MTTKRP partial Σ_k YV_k S_k, and Σ_k w_k w_kᵀ.  One CTA per slice
// (grid-stride), 256 threads; columns in chunks of 64: thread (jj, rg) owns
// column jc+jj and the rows r ≡ rg (mod 4).
constexpr int QZ_THREADS = 256;
constexpr int QZ_JC = 64;
constexpr int QZ_JC2 = 2 * QZ_JC;   // k_q_y: columns per pass (two per thread, QZ_JC apart)
constexpr int QZ_RC = 32;     // Q rows staged per pass

template <typename T>
__host__ __device__ inline size_t q_y_smem(int R) {
    const size_t RM = R <= 32 ? 32 : 64;
    return (RM * RM + (size_t)QZ_RC * RM + (size_t)QZ_JC2 * R + (size_t)R * (QZ_JC2 + 1)) * sizeof(T);
}

// n consecutive values from 16-byte aligned shared memory, as 16-byte loads.
template <int n>
__device__ __forceinline__ void ld_shared_vec(const float *p, float (&v)[n]) {
#pragma unroll
    for (int u = 0; u < n; u += 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p + u);
        v[u] = t.x; v[u + 1] = t.y; v[u + 2] = t.z; v[u + 3] = t.w;
    }
}
template <int n>
__device__ __forceinline__ void ld_shared_vec(const double *p, double (&v)[n]) {
#pragma unroll
    for (int u = 0; u < n; u += 2) {
        const double2 t = *reinterpret_cast<const double2 *>(p + u);
        v[u] = t.x; v[u + 1] = t.y;
    }
}

// The (r, s) pairs of an R×R result that the QZ_THREADS threads of a CTA
// split among themselves.  With R a multiple of 4, thread t owns runs of four
// consecutive s, s = 4·(t mod R/4) + i, in the rows r = ⌊t / (R/4)⌋ + g·ρ
// (ρ = ⌊QZ_THREADS / (R/4)⌋ rows per pass), pair index u = 4g + i; otherwise
// the pairs e = t + u·QZ_THREADS, r = e / R, s = e mod R.  False past the
// matrix.
__device__ __forceinline__ bool qz_pair(int R, int u, int &r, int &s) {
    const int t = threadIdx.x;
    if ((R & 3) == 0) {
        const int tpr = R >> 2, rpp = QZ_THREADS / tpr;
        r = t / tpr + (u >> 2) * rpp;
        s = ((t % tpr) << 2) + (u & 3);
        return t < tpr * rpp && r < R;
    }
    const int e = t + u * QZ_THREADS;
    r = e / R;
    s = e % R;
    return e < R * R;
}

// yv[u] += Σ_c Ys[r][c]·Vs[c][s] over one column chunk for the thread's pairs
// (qz_pair), each sum taken in c order in the product type.  Ys is R ×
// (QZ_JC + 1), Vs is QZ_JC × R; with R a multiple of 4 a run of four s is one
// vector load of the Vs row (16-byte aligned: the Vs base is, and the row
// pitch is R entries).
template <typename T, int NP>
__device__ __forceinline__ void qz_yv_chunk(const T *Ys, const T *Vs, int R, double (&yv)[NP],
                                            int ypitch = QZ_JC + 1) {
    const int t = threadIdx.x;
    if ((R & 3) == 0) {
        const int tpr = R >> 2, rpp = QZ_THREADS / tpr;
        if (t >= tpr * rpp) return;
        const int s0 = (t % tpr) << 2;
#pragma unroll
        for (int g = 0; g < NP / 4; ++g) {
            const int r = t / tpr + g * rpp;
            if (r < R) {
                T a[4] = {T(0), T(0), T(0), T(0)};
                for (int c = 0; c < QZ_JC; ++c) {
                    const T y = Ys[r * ypitch + c];
                    T v[4];
                    ld_shared_vec(Vs + c * R + s0, v);
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] += y * v[i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) yv[4 * g + i] += (double)a[i];
            }
        }
        return;
    }
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        int r, s2;
        if (qz_pair(R, u, r, s2)) {
            T a = T(0);
            for (int c = 0; c < QZ_JC; ++c) a += Ys[r * ypitch + c] * Vs[c * R + s2];
            yv[u] += (double)a;
        }
    }
}

template <typename TI, typename T, int RM>
__global__ void __launch_bounds__(QZ_THREADS, RM <= 32 ? 2 : 1) k_q_y(BatchDev b, QDev q, const TI *__restrict__ X,
                                                    const T *__restrict__ Qrows, T *__restrict__ Y,
                                                    const T *__restrict__ VT, double *__restrict__ MHpart,
                                                    double *__restrict__ WWpart) {
    extern __shared__ __align__(16) unsigned char qy_raw[];
    const int R = q.R, J = q.J, tid = threadIdx.x;
    T *Cs = reinterpret_cast<T *>(qy_raw);           // RM × RM  λ C_k (permuted, below)
    T *Qs = Cs + RM * RM;                            // QZ_RC × RM  Q rows (permuted)
    T *Vs = Qs + QZ_RC * RM;                         // QZ_JC2 × R
    T *Ys = Vs + QZ_JC2 * R;                         // R × (QZ_JC2 + 1)
    constexpr int YP = QZ_JC2 + 1;                   // Ys pitch
    const int jj = tid % QZ_JC, rg = tid / QZ_JC;
    const int nq = (R + 3) / 4;
    const bool lam_on = q.lam != 0.0;
    constexpr int NQ = RM / 4;                        // rows of Y per thread
    constexpr int NP = (RM * RM + QZ_THREADS - 1) / QZ_THREADS;   // (r, s) pairs per thread
    double mh[NP], ww[NP];
#pragma unroll
    for (int u = 0; u < NP; ++u) { mh[u] = 0.0; ww[u] = 0.0; }
    for (int k = blockIdx.x; k < b.K_all; k += gridDim.x) {
        const int t = b.tslot[k];
        T *Yk = Y + (int64_t)k * R * J;
        __syncthreads();
        // λC_k permuted so that a thread's NQ rows r = rg + 4u of column p are
        // contiguous: Cs[(p·4 + rg)·NQ + u] = λC_k[rg + 4u][p] (zero past R)
        for (int e = tid; e < RM * RM; e += QZ_THREADS) {
            const int p = e / RM, rg2 = (e % RM) / NQ, u = e % NQ;
            const int r = rg2 + 4 * u;
            Cs[e] = (!lam_on || r >= R || p >= R) ? T(0)
                                                        : (T)(q.lam * q.C[(int64_t)k * R * R + r * R + p]);
        }
        double yv[NP];
#pragma unroll
        for (int u = 0; u < NP; ++u) yv[u] = 0.0;
        // columns in passes of QZ_JC2: a thread owns columns j0 = jc + jj and
        // j1 = j0 + QZ_JC, each summed exactly as a single column would be
        for (int jc = 0; jc < J; jc += QZ_JC2) {
            const int j0 = jc + jj, j1 = j0 + QZ_JC;
            __syncthreads();
            // rows jc.. of Vᵀ's J×R layout are one contiguous block
            const int vlim = (J - jc < QZ_JC2 ? J - jc : QZ_JC2) * R;
            for (int e = tid; e < QZ_JC2 * R; e += QZ_THREADS) {
                Vs[e] = e < vlim ? VT[(int64_t)jc * R + e] : T(0);
            }
            // old Y chunk → Ys (all R rows, needed by every output row)
            for (int e = tid; e < R * QZ_JC2; e += QZ_THREADS) {
                const int r = e / QZ_JC2, c = e % QZ_JC2;
                Ys[r * YP + c] = (lam_on && jc + c < J) ? Yk[(int64_t)r * J + jc + c] : T(0);
            }
            __syncthreads();
            T acc[NQ], acc1[NQ];
#pragma unroll
            for (int u = 0; u < NQ; ++u) { acc[u] = T(0); acc1[u] = T(0); }
            for (int p = 0; p < R; ++p) {
                const T y = Ys[p * YP + jj], y1 = Ys[p * YP + jj + QZ_JC];
                T cv[NQ];
                ld_shared_vec(Cs + (p * 4 + rg) * NQ, cv);   // warp-uniform: broadcasts
#pragma unroll
                for (int u = 0; u < NQ; ++u) {
                    acc[u] += cv[u] * y;
                    acc1[u] += cv[u] * y1;
                }
            }
            if (t >= 0) {
                for (int si = b.tseg_ptr[t]; si < b.tseg_ptr[t + 1]; ++si) {
                    const int sg = b.tseg_idx[si];
                    const int64_t r0 = b.seg_row[sg], r1 = b.seg_row[sg + 1];
                    for (int64_t c0 = r0; c0 < r1; c0 += QZ_RC) {
                        const int nr = (int)(r1 - c0 < QZ_RC ? r1 - c0 : QZ_RC);
                        __syncthreads();
                        // the same permutation: Qs[(i·4 + rg)·NQ + u] = Q(c0 + i, rg + 4u)
                        for (int e = tid; e < nr * RM; e += QZ_THREADS) {
                            const int i = e / RM, rg2 = (e % RM) / NQ, u = e % NQ;
                            const int r = rg2 + 4 * u;
                            Qs[e] = r < R ? Qrows[(c0 + i) * R + r] : T(0);
                        }
                        __syncthreads();
                        if (j0 < J) {
                            // four rows' loads in flight at a time, both columns
                            const TI *xb = X + c0 * J;
                            const bool on1 = j1 < J;
                            for (int i0 = 0; i0 < nr; i0 += 4) {
                                T xv[4], xw[4];
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    const bool in = i0 + i < nr;
                                    xv[i] = in ? (T)xb[(int64_t)(i0 + i) * J + j0] : T(0);
                                    xw[i] = in && on1 ? (T)xb[(int64_t)(i0 + i) * J + j1] : T(0);
                                }
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    if (i0 + i < nr) {
                                        T qv[NQ];
                                        ld_shared_vec(Qs + ((i0 + i) * 4 + rg) * NQ, qv);
#pragma unroll
                                        for (int u = 0; u < NQ; ++u) {
                                            acc[u] += qv[u] * xv[i];
                                            acc1[u] += qv[u] * xw[i];
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                const int r = rg + 4 * u;
                if (u < nq && r < R) {
                    if (j0 < J) Yk[(int64_t)r * J + j0] = acc[u];
                    if (j1 < J) Yk[(int64_t)r * J + j1] = acc1[u];
                    Ys[r * YP + jj] = j0 < J ? acc[u] : T(0);
                    Ys[r * YP + jj + QZ_JC] = j1 < J ? acc1[u] : T(0);
                }
            }
            __syncthreads();
            // YV partial, one sum per half of the pass (as per QZ_JC-column
            // chunk): thread owns pairs (r, s)
            qz_yv_chunk(Ys, Vs, R, yv, YP);
            if (jc + QZ_JC < J) qz_yv_chunk(Ys + QZ_JC, Vs + QZ_JC * R, R, yv, YP);
        }
        const double *wk = q.W + (int64_t)k * R;
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            int r, s2;
            if (qz_pair(R, u, r, s2)) {
                mh[u] += yv[u] * wk[s2];
                ww[u] += wk[r] * wk[s2];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        int r, s2;
        if (qz_pair(R, u, r, s2)) {
            MHpart[(int64_t)blockIdx.x * R * R + r * R + s2] = mh[u];
            WWpart[(int64_t)blockIdx.x * R * R + r * R + s2] = ww[u];
        }
    }
}

// Sums of per-CTA FP64 partials, in place: parts[e] = Σ_{p < nb} parts[p·n + e]
// for e < n, each entry by one thread in the order p = 0, 1, ... (so the
// result has the bits of a sequential sum).  Entry e is read and written by
// its own thread only, so the in-place write is race-free.
static __global__ void k_q_psum(double *__restrict__ parts, int nb, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int p = 0; p < nb; ++p) a += parts[(int64_t)p * n + e];
        parts[e] = a;
    }
}

// H = MH (Γ ∗ WᵀW)⁺ and PV = (HᵀH ∗ WᵀW)⁺, one warp; WW (R×R) is kept.
static __global__ void k_q_h(const double *__restrict__ MHpart, const double *__restrict__ WWpart, int nb,
                      QDev q, double *__restrict__ WW, double *__restrict__ PV) {
    extern __shared__ double hs[];
    const int R = q.R, ld = q_ld(R), lane = threadIdx.x & 31;
    double *MH = hs, *A = MH + R * ld, *E = A + R * ld, *O = E + R * ld, *f = O + R * ld;
    for (int e = lane; e < R * R; e += 32) {
        double m = 0.0, ww = 0.0;
        for (int p = 0; p < nb; ++p) {
            m += MHpart[(int64_t)p * R * R + e];
            ww += WWpart[(int64_t)p * R * R + e];
        }
        MH[(e / R) * ld + (e % R)] = m;
        WW[e] = ww;
        A[(e / R) * ld + (e % R)] = q.Gam[e] * ww;
    }
    __syncwarp();
    warp_psd_pinv(A, E, f, O, R, ld, q.rtol, 1, true);
    // H = MH O
    for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, s = e % R;
        double a = 0.0;
        for (int p = 0; p < R; ++p) a += MH[r * ld + p] * O[p * ld + s];
        E[r * ld + s] = a;
    }
    __syncwarp();
    for (int e = lane; e < R * R; e += 32) q.H[e] = E[(e / R) * ld + (e % R)];
    __syncwarp();
    // PV = (HᵀH ∗ WᵀW)⁺
    for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, s = e % R;
        double a = 0.0;
        for (int p = 0; p < R; ++p) a += E[p * ld + r] * E[p * ld + s];
        A[r * ld + s] = a * WW[e];
    }
    __syncwarp();
    warp_psd_pinv(A, MH, f, O, R, ld, q.rtol, 1, true);
    for (int e = lane; e < R * R; e += 32) PV[e] = O[(e / R) * ld + (e % R)];
}

// V-MTTKRP: slot_b[j][s] = Σ_{k in CTA b} w_k[s] Σ_r Y_k[r][j] H[r][s]
// (= Σ_k Y_kᵀ H S_k).  A thread owns column j of every slice of its CTA and
// keeps its R accumulators in registers across those slices; H sits in
// shared memory, and Y_k's column j is read coalesced across the threads.
constexpr int QV_THREADS = 128;

template <typename T, int RM>
__global__ void __launch_bounds__(QV_THREADS) k_q_vpart(int K_all, QDev q, const T *__restrict__ Y,
                                                        double *__restrict__ slots) {
    __shared__ __align__(16) T Hs[RM * RM];           // H, row pitch RM, zero-padded
    const int R = q.R, J = q.J, tid = threadIdx.x, lane = tid & 31;
    for (int e = tid; e < RM * RM; e += QV_THREADS) {
        const int r = e / RM, s2 = e % RM;
        Hs[e] = (r < R && s2 < R) ? (T)q.H[r * R + s2] : T(0);
    }
    __syncthreads();
    double *sl = slots + (size_t)blockIdx.x * J * R;
    // every lane of a warp takes every column pass (the weights are shared by
    // shuffles); lanes past J only skip their loads and stores
    for (int j0 = 0; j0 < J; j0 += QV_THREADS) {
        const int j = j0 + tid;
        const bool on = j < J;
        T acc[RM];
#pragma unroll
        for (int s2 = 0; s2 < RM; ++s2) acc[s2] = T(0);
        for (int k = blockIdx.x; k < K_all; k += gridDim.x) {
            const T *Yk = Y + (int64_t)k * R * J + (on ? j : 0);
            // w_k in the product type, entry s on lane s mod 32 (converted once)
            const double *wk = q.W + (int64_t)k * R;
            const T w0 = lane < R ? (T)wk[lane] : T(0);
            const T w1 = (RM > 32 && lane + 32 < R) ? (T)wk[lane + 32] : T(0);
            T t[RM];
#pragma unroll
            for (int s2 = 0; s2 < RM; ++s2) t[s2] = T(0);
            for (int r = 0; r < R; ++r) {
                const T y = on ? Yk[(int64_t)r * J] : T(0);
#pragma unroll
                for (int s0 = 0; s0 < RM; s0 += 4) {
                    T h[4];
                    ld_shared_vec(Hs + r * RM + s0, h);
#pragma unroll
                    for (int i = 0; i < 4; ++i) t[s0 + i] += y * h[i];
                }
            }
#pragma unroll
            for (int s2 = 0; s2 < RM; ++s2) {
                const T w = __shfl_sync(0xffffffffu, s2 < 32 ? w0 : w1, s2 & 31);
                if (s2 < R) acc[s2] += w * t[s2];
            }
        }
        if (on) {
#pragma unroll
            for (int s2 = 0; s2 < RM; ++s2)
                if (s2 < R) sl[(int64_t)j * R + s2] = (double)acc[s2];
        }
    }
}

// V = (Σ slots) PV, one warp per row j; V in the product type refreshed.
template <typename T>
__global__ void k_q_v(const double *__restrict__ slots, int nb, const double *__restrict__ PV, int J,
                      int R, double *__restrict__ V, T *__restrict__ VT) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= J) return;
    for (int s = lane; s < R; s += 32) {
        double v = 0.0;
        for (int r = 0; r < R; ++r) {
            double m = 0.0;
            for (int p = 0; p < nb; ++p) m += slots[(size_t)p * J * R + (int64_t)j * R + r];
            v += m * PV[r * R + s];
        }
        V[(int64_t)j * R + s] = v;
        VT[(int64_t)j * R + s] = (T)v;
    }
}

// PW = (HᵀH ∗ VᵀV)⁺ with the new H and V (one warp).
static __global__ void k_q_pw(QDev q, double *__restrict__ PW) {
    extern __shared__ double ws[];
    const int R = q.R, ld = q_ld(R), lane = threadIdx.x & 31;
    double *A = ws, *E = A + R * ld, *O = E + R * ld, *f = O + R * ld;
    for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, s = e % R;
        double a = 0.0;
        for (int p = 0; p < R; ++p) a += q.H[p * R + r] * q.H[p * R + s];
        A[r * ld + s] = a * q.Gam[e];
    }
    __syncwarp();
    warp_psd_pinv(A, E, f, O, R, ld, q.rtol, 1, true);
    for (int e = lane; e < R * R; e += 32) PW[e] = O[(e / R) * ld + (e % R)];
}

// W(k,:) = u PW with u_r = (Hᵀ Y_k V)[r][r] = Σ_q H[q][r] (Y_k V)[q][r].
// One CTA per slice; Y_k V in column chunks.
template <typename T>
__host__ __device__ inline size_t q_w_smem(int R) {
    return ((size_t)QZ_JC2 * R + (size_t)R * (QZ_JC2 + 1)) * sizeof(T) + (size_t)(64 + R * R) * 8 + 16;
}

template <typename T>
__global__ void __launch_bounds__(QZ_THREADS) k_q_w(int K_all, QDev q, const T *__restrict__ Y,
                                                    const T *__restrict__ VT,
                                                    const double *__restrict__ PW) {
    extern __shared__ __align__(16) unsigned char qw_raw[];
    const int R = q.R, J = q.J, tid = threadIdx.x;
    constexpr int YP = QZ_JC2 + 1;                    // Ys pitch
    T *Vs = reinterpret_cast<T *>(qw_raw);            // QZ_JC2 × R
    T *Ys = Vs + QZ_JC2 * R;                          // R × (QZ_JC2 + 1)
    const size_t off = (((size_t)QZ_JC2 * R + (size_t)R * YP) * sizeof(T) + 15) / 16 * 16;
    double *u = reinterpret_cast<double *>(qw_raw + off);   // 64
    double *red = u + 64;                                   // R × R
    for (int k = blockIdx.x; k < K_all; k += gridDim.x) {
        const T *Yk = Y + (int64_t)k * R * J;
        double yv[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) yv[v] = 0.0;
        // passes of QZ_JC2 columns, summed per half (QZ_JC columns) as before
        for (int jc = 0; jc < J; jc += QZ_JC2) {
            __syncthreads();
            // rows jc.. of Vᵀ's J×R layout are one contiguous block
            const int vlim = (J - jc < QZ_JC2 ? J - jc : QZ_JC2) * R;
            for (int e = tid; e < QZ_JC2 * R; e += QZ_THREADS) {
                Vs[e] = e < vlim ? VT[(int64_t)jc * R + e] : T(0);
            }
            for (int e = tid; e < R * QZ_JC2; e += QZ_THREADS) {
                const int r = e / QZ_JC2, c = e % QZ_JC2;
                Ys[r * YP + c] = jc + c < J ? Yk[(int64_t)r * J + jc + c] : T(0);
            }
            __syncthreads();
            qz_yv_chunk(Ys, Vs, R, yv, YP);
            if (jc + QZ_JC < J) qz_yv_chunk(Ys + QZ_JC, Vs + QZ_JC * R, R, yv, YP);
        }
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            int r, s;
            if (qz_pair(R, v, r, s)) red[r * R + s] = q.H[r * R + s] * yv[v];
        }
        __syncthreads();
        for (int r = tid; r < R; r += QZ_THREADS) {
            double a = 0.0;
            for (int p = 0; p < R; ++p) a += red[p * R + r];
            u[r] = a;
        }
        __syncthreads();
        for (int s = tid; s < R; s += QZ_THREADS) {
            double a = 0.0;
            for (int r = 0; r < R; ++r) a += u[r] * PW[r * R + s];
            q.W[(int64_t)k * R + s] = a;
        }
    }
}

// The squared residual of X_new against Q_new H S_k Vᵀ with the updated
// factors.  Vᵀ (R×Jc, product type) is staged in shared memory one column
// chunk of Jc (a multiple of 128) at a time; one warp per row forms
// z = q H S_k and x̂ = z Vᵀ four columns at a time (lane l owns columns
// 4l + 128m of the chunk), then Σ (x − x̂)² and Σ x².  Per-CTA partials of
// (Σ residual², Σ ‖x‖²).
template <typename T>
__host__ __device__ inline int q_out_chunk(int R, int J) {
    const int Jp = ((J + 127) / 128) * 128;
    int cap = (int)((190 * 1024 - (size_t)R * R * sizeof(T)) / ((size_t)R * sizeof(T)) / 128) * 128;
    if (cap < 128) cap = 128;
    return Jp < cap ? Jp : cap;
}
template <typename T>
__host__ __device__ inline size_t q_out_smem(int R, int J) {
    return ((size_t)R * q_out_chunk<T>(R, J) + 8 * 64 + (size_t)R * R) * sizeof(T);
}

template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_q_out(int64_t N, QDev q, const int *__restrict__ row_slice,
                                               const TI *__restrict__ X, const T *__restrict__ Qrows,
                                               const T *__restrict__ VT, double *__restrict__ fitpart) {
    extern __shared__ unsigned char qo_raw[];
    const int R = q.R, J = q.J;
    const int Jc = q_out_chunk<T>(R, J);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *Vt = reinterpret_cast<T *>(qo_raw);                     // R × Jc, Vt[s][j] = V[j0 + j][s]
    T *zs = Vt + (size_t)R * Jc + (size_t)wid * 64;            // per warp z
    T *Hs = Vt + (size_t)R * Jc + 8 * 64;                      // H in the product type
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Hs[e] = (T)q.H[e];
    double res = 0.0, xn = 0.0;
    for (int jb = 0; jb < J; jb += Jc) {
        __syncthreads();
        for (int e = threadIdx.x; e < R * Jc; e += blockDim.x) {
            const int s2 = e / Jc, j = jb + e % Jc;
            Vt[e] = j < J ? VT[(int64_t)j * R + s2] : T(0);
        }
        __syncthreads();
        for (int64_t row = (int64_t)blockIdx.x * nw + wid; row < N; row += (int64_t)gridDim.x * nw) {
            const int k = row_slice[row];
            __syncwarp();
            // z = q H S_k: the row's q entries read once (lane l holds q_l and
            // q_{l+32}) and broadcast by shuffles
            {
                const T qa = lane < R ? Qrows[row * R + lane] : T(0);
                const T qb = lane + 32 < R ? Qrows[row * R + lane + 32] : T(0);
                T a0 = T(0), a1 = T(0);
                for (int r = 0; r < R; ++r) {
                    const T qr = __shfl_sync(0xffffffffu, r < 32 ? qa : qb, r & 31);
                    if (lane < R) a0 += qr * Hs[r * R + lane];
                    if (lane + 32 < R) a1 += qr * Hs[r * R + lane + 32];
                }
                if (lane < R) zs[lane] = a0 * (T)q.W[(int64_t)k * R + lane];
                if (lane + 32 < R) zs[lane + 32] = a1 * (T)q.W[(int64_t)k * R + lane + 32];
            }
            __syncwarp();
            const TI *xr = X + row * J + jb;
            // FP32 data and products: the lane's share of the row is summed in
            // double-float (x − x̂ exactly by TwoSum, each square split by
            // TwoProduct, each addition by TwoSum) and added to the FP64 totals
            // once per row, so the FP64 pipe sees four additions per row, not
            // five operations per entry
            constexpr bool f32 = std::is_same<T, float>::value && std::is_same<TI, float>::value;
            df rs = {0.f, 0.f}, xs = {0.f, 0.f};
            for (int j0 = 4 * lane; j0 < Jc && jb + j0 < J; j0 += 128) {
                T h0 = T(0), h1 = T(0), h2 = T(0), h3 = T(0);
                for (int s2 = 0; s2 < R; ++s2) {
                    const T z = zs[s2];
                    const T *v = Vt + (size_t)s2 * Jc + j0;
                    h0 += z * v[0];
                    h1 += z * v[1];
                    h2 += z * v[2];
                    h3 += z * v[3];
                }
                const T hh[4] = {h0, h1, h2, h3};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jb + j0 + u < J) {
                        if constexpr (f32) {
                            const float x = (float)xr[j0 + u];
                            const df d = two_sum(x, -(float)hh[u]);     // x − x̂ exactly
                            const df p = two_prod(d.hi, d.hi);
                            const df t = two_sum(rs.hi, p.hi);
                            rs = {t.hi, __fadd_rn(rs.lo, __fadd_rn(t.lo, fmaf(2.f * d.hi, d.lo, p.lo)))};
                            const df px = two_prod(x, x);
                            const df tx = two_sum(xs.hi, px.hi);
                            xs = {tx.hi, __fadd_rn(xs.lo, __fadd_rn(tx.lo, px.lo))};
                        } else {
                            const double x = (double)xr[j0 + u];
                            const double d = x - (double)hh[u];
                            res += d * d;
                            xn += x * x;
                        }
                    }
                }
            }
            if constexpr (f32) {
                res += (double)rs.hi + (double)rs.lo;
                xn += (double)xs.hi + (double)xs.lo;
            }
        }
    }
    res = warp_sum(res);
    xn = warp_sum(xn);
    __shared__ double red[2][32];
    if (lane == 0) {
        red[0][wid] = res;
        red[1][wid] = xn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) {
            a += red[0][w2];
            c += red[1][w2];
        }
        fitpart[2 * blockIdx.x] = a;
        fitpart[2 * blockIdx.x + 1] = c;
    }
}

static __global__ void k_q_fit(const double *__restrict__ fitpart, int nb, const int *__restrict__ gam_ok,
                        double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    double a = 0.0, c = 0.0;
    for (int p = lane; p < nb; p += 32) {
        a += fitpart[2 * p];
        c += fitpart[2 * p + 1];
    }
    a = warp_sum(a);
    c = warp_sum(c);
    if (lane == 0) {
        out[0] = c > 0.0 ? 1.0 - sqrt(a / c) : 1.0;
        out[1] = c;
        out[2] = a;
        out[3] = (double)*gam_ok;
    }
}

}  // namespace dash
