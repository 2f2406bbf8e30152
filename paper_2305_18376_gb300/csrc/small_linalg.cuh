// Warp-level FP64 routines for the small R×R systems of the Dash update:
// (S_k VᵀV S_k)⁺ (Lemma 1, Eq. 11), (VᵀV ∗ D_k)⁺ (Lemma 2, Eq. 12), G⁺
// (Lemma 3, Eq. 17) and, in mode Q, B_k^{-1/2}.
//
// All matrices live in shared memory, row-major with leading dimension ld,
// and are handled by one warp (R <= 64, so each lane owns at most two rows).
// "⁺" is the Moore-Penrose pseudo-inverse of a symmetric PSD matrix:
// eigenvalues <= rtol · max|eigenvalue| count as zero.  The fast path is a
// Cholesky factorisation, taken only when every pivot is far above that
// cut-off; otherwise a cyclic Jacobi eigen-decomposition gives the exact
// pseudo-inverse.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace dash {

constexpr int kMaxR = 64;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// In-place lower Cholesky A = L Lᵀ of an n×n SPD matrix (lower triangle of A
// is overwritten by L; the strict upper triangle is left untouched).
// Returns false as soon as a pivot is not above `tol` (also for NaN).
__device__ inline bool warp_cholesky(double *A, int n, int ld, double tol) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; ++j) {
        __syncwarp();
        const double d = A[j * ld + j];
        if (!(d > tol)) return false;
        const double l = sqrt(d);
        const double inv = 1.0 / l;
        for (int i = j + 1 + lane; i < n; i += 32) A[i * ld + j] *= inv;
        __syncwarp();
        if (lane == 0) A[j * ld + j] = l;
        for (int i = j + 1 + lane; i < n; i += 32) {
            const double lij = A[i * ld + j];
            for (int k = j + 1; k <= i; ++k) A[i * ld + k] -= lij * A[k * ld + j];
        }
    }
    __syncwarp();
    return true;
}

// Solve L Lᵀ x = b with L from warp_cholesky; b (length n, shared) is
// overwritten by x.
__device__ inline void warp_cholesky_solve(const double *L, int n, int ld, double *b) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; ++j) {
        __syncwarp();
        const double yj = b[j] / L[j * ld + j];
        __syncwarp();
        if (lane == 0) b[j] = yj;
        for (int i = j + 1 + lane; i < n; i += 32) b[i] -= L[i * ld + j] * yj;
    }
    for (int j = n - 1; j >= 0; --j) {
        __syncwarp();
        const double xj = b[j] / L[j * ld + j];
        __syncwarp();
        if (lane == 0) b[j] = xj;
        for (int i = lane; i < j; i += 32) b[i] -= L[j * ld + i] * xj;
    }
    __syncwarp();
}

// Cyclic Jacobi eigen-decomposition of a symmetric n×n matrix.  On return
// the diagonal of A holds the eigenvalues and the columns of E the
// eigenvectors (A_in = E diag(A_out) Eᵀ).  Off-diagonal entries of A are
// destroyed.  Rotations follow the symmetric Schur 2×2 step of Golub and
// Van Loan (Matrix Computations, §8.5).
//
// A pair (p, q) is rotated only while |a_pq| > 1e-15·sqrt(|a_pp a_qq|), the
// relative threshold of Demmel and Veselić ("Jacobi's method is more
// accurate than QR", SIAM J. Matrix Anal. Appl. 13, 1992), which stops at
// rounding level; and not when both a_pp and a_qq are below tiny_abs (for a
// PSD matrix |a_pq| <= sqrt(a_pp a_qq) then, so the pair's eigenvalues stay
// below 2·tiny_abs: callers pass a quarter of their pseudo-inverse cut, and
// such a pair is dropped whichever way it is rotated).  The sweeps stop at
// the first one that rotates nothing.  A threshold below the unit roundoff
// never stops on a rank-deficient matrix: the rotations keep refilling the
// zeroed entries at rounding level.
__device__ inline void warp_jacobi_eig(double *A, double *E, int n, int ld, double tiny_abs = 0.0,
                                       int max_sweeps = 50) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < n * n; i += 32) {
        const int r = i / n, c = i % n;
        E[r * ld + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = lane; i < n * n; i += 32) {
            const int r = i / n, c = i % n;
            const double v = A[r * ld + c];
            if (r == c) dia += v * v; else off += v * v;
        }
        off = warp_sum(off);
        dia = warp_sum(dia);
        if (off <= 1e-32 * dia || off == 0.0) break;
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                __syncwarp();
                const double apq = A[p * ld + q];
                const double app = A[p * ld + p];
                const double aqq = A[q * ld + q];
                if (fabs(apq) <= 1e-300 ||
                    fabs(apq) <= 1e-15 * sqrt(fabs(app) * fabs(aqq)) ||
                    (fabs(app) <= tiny_abs && fabs(aqq) <= tiny_abs)) {
                    continue;
                }
                ++rotated;
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) /
                                 (fabs(theta) + sqrt(1.0 + theta * theta));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                __syncwarp();
                for (int k = lane; k < n; k += 32) {
                    if (k != p && k != q) {
                        const double akp = A[k * ld + p], akq = A[k * ld + q];
                        const double nkp = c * akp - s * akq;
                        const double nkq = s * akp + c * akq;
                        A[k * ld + p] = nkp; A[p * ld + k] = nkp;
                        A[k * ld + q] = nkq; A[q * ld + k] = nkq;
                    }
                    const double ekp = E[k * ld + p], ekq = E[k * ld + q];
                    E[k * ld + p] = c * ekp - s * ekq;
                    E[k * ld + q] = s * ekp + c * ekq;
                }
                if (lane == 0) {
                    A[p * ld + p] = app - t * apq;
                    A[q * ld + q] = aqq + t * apq;
                    A[p * ld + q] = 0.0;
                    A[q * ld + p] = 0.0;
                }
            }
        }
        __syncwarp();
        if (rotated == 0) break;
    }
    __syncwarp();
}

// Spectral weights f(μ_i) after warp_jacobi_eig: power 1 → 1/μ, power 2 →
// 1/sqrt(μ); eigenvalues <= rtol·max|μ| (and all of them when max|μ| = 0)
// get weight 0.  f has length n (shared).
__device__ inline void warp_spectral_weights(const double *A, int n, int ld, double rtol,
                                             int power, double *f) {
    const int lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int i = lane; i < n; i += 32) mx = fmax(mx, fabs(A[i * ld + i]));
    mx = warp_max(mx);
    const double cut = rtol * mx;
    for (int i = lane; i < n; i += 32) {
        const double mu = A[i * ld + i];
        double v = 0.0;
        if (mx > 0.0 && mu > cut) v = (power == 1) ? 1.0 / mu : 1.0 / sqrt(mu);
        f[i] = v;
    }
    __syncwarp();
}

// out = E diag(f) Eᵀ (n×n, shared, may not alias E).
__device__ inline void warp_spectral_apply(const double *E, const double *f, int n, int ld,
                                           double *out) {
    const int lane = threadIdx.x & 31;
    for (int idx = lane; idx < n * n; idx += 32) {
        const int r = idx / n, c = idx % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += E[r * ld + k] * f[k] * E[c * ld + k];
        out[r * ld + c] = s;
    }
    __syncwarp();
}

// Inverse of an SPD matrix from its Cholesky factor (lower triangle of L,
// as left by warp_cholesky): lane c solves L Lᵀ x = e_c for column c of the
// inverse on its own, with the reciprocals of diag(L) computed once, so the
// inner loops need no divisions and no warp synchronisation (FP64 division
// is a long software sequence on parts with a slow FP64 pipe).  out must not
// alias L; rinv is length-n workspace.  n <= 64.
__device__ inline void warp_cholesky_inverse(const double *L, int n, int ld, double *out,
                                             double *rinv) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < n; i += 32) rinv[i] = 1.0 / L[i * ld + i];
    __syncwarp();
    for (int c = lane; c < n; c += 32) {
        // forward: L y = e_c (y[i] = 0 for i < c); y kept in column c of out
        for (int i = 0; i < c; ++i) out[i * ld + c] = 0.0;
        for (int i = c; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[i * ld + k] * out[k * ld + c];
            out[i * ld + c] = s * rinv[i];
        }
        // backward: Lᵀ x = y
        for (int i = n - 1; i >= 0; --i) {
            double s = out[i * ld + c];
            for (int k = i + 1; k < n; ++k) s -= L[k * ld + i] * out[k * ld + c];
            out[i * ld + c] = s * rinv[i];
        }
    }
    __syncwarp();
}

// Pseudo-inverse (power 1) or pseudo-inverse square root (power 2) of the
// symmetric PSD matrix in A, written to out.  A and E are destroyed (E is
// workspace), f is length-n workspace.  When `try_cholesky` and power == 1,
// a Cholesky inverse is used if every pivot exceeds 100·rtol·max(diag).
__device__ inline void warp_psd_pinv(double *A, double *E, double *f, double *out, int n,
                                     int ld, double rtol, int power, bool try_cholesky) {
    const int lane = threadIdx.x & 31;
    double md = 0.0;
    for (int i = lane; i < n; i += 32) md = fmax(md, fabs(A[i * ld + i]));
    md = warp_max(md);
    if (power == 1 && try_cholesky) {
        for (int i = lane; i < n * n; i += 32) E[(i / n) * ld + (i % n)] = A[(i / n) * ld + (i % n)];
        __syncwarp();
        if (md > 0.0 && warp_cholesky(E, n, ld, 100.0 * rtol * md)) {
            warp_cholesky_inverse(E, n, ld, out, f);
            // symmetrise
            for (int idx = lane; idx < n * n; idx += 32) {
                const int r = idx / n, c = idx % n;
                if (r < c) {
                    const double v = 0.5 * (out[r * ld + c] + out[c * ld + r]);
                    out[r * ld + c] = v;
                    out[c * ld + r] = v;
                }
            }
            __syncwarp();
            return;
        }
    }
    // both powers drop the eigenvalues <= rtol·max
    warp_jacobi_eig(A, E, n, ld, 0.25 * rtol * md);
    warp_spectral_weights(A, n, ld, rtol, power, f);
    warp_spectral_apply(E, f, n, ld, out);
}

// x = A⁺ b for symmetric PSD A: Cholesky when all pivots exceed
// 100·rtol·max(diag), else Jacobi pseudo-inverse.  A is destroyed; L and E
// are n×ld workspaces; b (shared, length n) is overwritten with x; f is
// length-n workspace.  Returns 0 for the Cholesky path, 1 for the eigen path.
__device__ inline int warp_psd_solve(double *A, double *L, double *E, double *b, double *f,
                                     int n, int ld, double rtol) {
    const int lane = threadIdx.x & 31;
    double md = 0.0;
    for (int i = lane; i < n; i += 32) md = fmax(md, fabs(A[i * ld + i]));
    md = warp_max(md);
    for (int i = lane; i < n * n; i += 32) L[(i / n) * ld + (i % n)] = A[(i / n) * ld + (i % n)];
    __syncwarp();
    if (md > 0.0 && warp_cholesky(L, n, ld, 100.0 * rtol * md)) {
        warp_cholesky_solve(L, n, ld, b);
        return 0;
    }
    warp_jacobi_eig(A, E, n, ld, 0.25 * rtol * md);
    warp_spectral_weights(A, n, ld, rtol, 1, f);
    // x = E diag(f) Eᵀ b, using L's first row as scratch for y = Eᵀ b
    double *y = L;
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += E[i * ld + k] * b[i];
        y[k] = s * f[k];
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += E[i * ld + k] * y[k];
        f[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) b[i] = f[i];
    __syncwarp();
    return 1;
}

}  // namespace dash
