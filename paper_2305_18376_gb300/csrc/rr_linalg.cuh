// Warp-level R×R linear algebra for the constrained-mode summaries, written
// once for two scalar types: double (FP64 path) and df (double-float pairs,
// mixed path; GB300 runs FP64 at about 1/57 of the FP32 rate, and df keeps
// about 44 bits at a fraction of the FP64 cost).
//
//   warp_qr_append        L ← R factor of [L; A]: Householder reflections that
//                         fold m ≤ 32 new rows into an upper-triangular L
//   warp_eig_factor       eigenbasis and eigenvalues of LᵀL from L, without
//                         forming LᵀL in a bad basis; warp_sqrt_weights and
//                         warp_spectral_s then give (LᵀL)^{∓1/2}
//
// Why not eig(LᵀL) directly: B = LᵀL has the squared condition number of the
// stacked A rows, and on the planted workloads cond(B) reaches 1e9-1e12, so
// any eigen-solver that sees B in the standard basis loses that many digits
// of its small eigenvalues.  Instead each pass forms G = L·E in the current
// eigenbasis estimate E and runs cyclic Jacobi on M = GᵀG.  Once E is close,
// M is nearly diagonal after diagonal scaling, and Jacobi on such a matrix
// determines every eigenvalue to high relative accuracy (Demmel and Veselić,
// "Jacobi's method is more accurate than QR", 1992); forming M = GᵀG adds
// only scaled errors |δM_ij| <= γ·sqrt(M_ii M_jj), which that analysis
// tolerates.  A cold start (E = I) takes two passes; a warm start from the
// previous update's basis usually converges in the first sweeps of each.
//
// Rotation angles are computed in FP32 (they need only be close, not exact)
// and turned into an exactly orthogonal pair c = 1/sqrt(1 + t²), s = c·t in
// the working type, so no FP64 division or square root sits in the inner
// loop.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "df.cuh"

namespace dash {

template <class S> struct RT;

template <> struct RT<double> {
    static __device__ __forceinline__ bool invertible(double a) { return fabs(a) > 1e-290; }
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double one() { return 1.0; }
    static __device__ __forceinline__ double from_d(double x) { return x; }
    static __device__ __forceinline__ double from_f(float x) { return (double)x; }
    static __device__ __forceinline__ double to_d(double a) { return a; }
    static __device__ __forceinline__ float hi(double a) { return (float)a; }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double mulf(double a, float b) { return a * (double)b; }
    static __device__ __forceinline__ double fma(double acc, double a, double b) { return ::fma(a, b, acc); }
    static __device__ __forceinline__ double sqrt_(double a) { return a > 0.0 ? ::sqrt(a) : 0.0; }
    static __device__ __forceinline__ double rsqrt_(double a) { return a > 0.0 ? ::rsqrt(a) : 0.0; }
    static __device__ __forceinline__ double recip(double a) { return 1.0 / a; }
    static __device__ __forceinline__ double shfl_xor(double a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
};

template <> struct RT<float> {
    static __device__ __forceinline__ bool invertible(float a) { return fabsf(a) > 1e-30f; }
    static __device__ __forceinline__ float zero() { return 0.f; }
    static __device__ __forceinline__ float one() { return 1.f; }
    static __device__ __forceinline__ float from_d(double x) { return (float)x; }
    static __device__ __forceinline__ float from_f(float x) { return x; }
    static __device__ __forceinline__ double to_d(float a) { return (double)a; }
    static __device__ __forceinline__ float hi(float a) { return a; }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float mulf(float a, float b) { return a * b; }
    static __device__ __forceinline__ float fma(float acc, float a, float b) { return fmaf(a, b, acc); }
    static __device__ __forceinline__ float sqrt_(float a) { return a > 0.f ? sqrtf(a) : 0.f; }
    // rsqrtf refined by one Newton step (about 1 ulp): rotations built from
    // it stay orthogonal to FP32 round-off
    static __device__ __forceinline__ float rsqrt_(float a) {
        if (!(a > 0.f)) return 0.f;
        const float y = rsqrtf(a);
        return y * fmaf(-0.5f * a * y, y, 1.5f);
    }
    static __device__ __forceinline__ float recip(float a) { return 1.f / a; }
    static __device__ __forceinline__ float shfl_xor(float a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
};

template <> struct RT<df> {
    // FP32 exponent range: keep the reciprocal (and its Newton step) normal
    static __device__ __forceinline__ bool invertible(df a) { return fabsf(a.hi) > 1e-30f; }
    static __device__ __forceinline__ df zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ df one() { return {1.f, 0.f}; }
    static __device__ __forceinline__ df from_d(double x) { return df_from_double(x); }
    static __device__ __forceinline__ df from_f(float x) { return {x, 0.f}; }
    static __device__ __forceinline__ double to_d(df a) { return df_to_double(a); }
    static __device__ __forceinline__ float hi(df a) { return a.hi; }
    static __device__ __forceinline__ df add(df a, df b) { return df_add(a, b); }
    static __device__ __forceinline__ df sub(df a, df b) { return df_sub(a, b); }
    static __device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }
    static __device__ __forceinline__ df mulf(df a, float b) { return df_mul_f(a, b); }
    static __device__ __forceinline__ df fma(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }
    static __device__ __forceinline__ df sqrt_(df a) { return df_sqrt(a); }
    static __device__ __forceinline__ df rsqrt_(df a) { return df_rsqrt(a); }
    static __device__ __forceinline__ df recip(df a) { return df_recip(a); }
    static __device__ __forceinline__ df shfl_xor(df a, int m) {
        return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
    }
};

template <class S> __device__ __forceinline__ S warp_sum_s(S v) {
    using O = RT<S>;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = O::add(v, O::shfl_xor(v, m));
    return v;
}

// L (R×R upper-triangular, non-negative diagonal, shared, leading dimension
// ld) ← the R factor of [L; A] with A the m ≤ 32 rows at A (shared, lda).
// A is destroyed.  One Householder reflection per column j maps
// (L[j][j], A[0..m-1][j]) to (‖·‖, 0); row j is then negated so the diagonal
// stays non-negative (a sign flip of one row is itself orthogonal).
template <class S>
__device__ void warp_qr_append(S *L, int ld, S *A, int lda, int m, int R) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < R; ++j) {
        const S aij = lane < m ? A[lane * lda + j] : O::zero();
        const S sq = warp_sum_s(O::mul(aij, aij));
        const S ljj = L[j * ld + j];
        __syncwarp();
        const S alpha = O::sqrt_(O::fma(sq, ljj, ljj));
        const S v0 = O::add(ljj, alpha);                     // ljj >= 0: no cancellation
        const S av = O::mul(alpha, v0);
        // nothing below the diagonal (sq = 0), or only residues so small that
        // vᵀv/2 is not invertible in the working type (the column of a
        // rank-deficient slice after its rank is reached): no reflection
        if (O::hi(sq) != 0.f && O::invertible(av)) {
            const S tau = O::recip(av);                        // 2 / vᵀv
            for (int c = j + 1 + lane; c < R; c += 32) {
                S d = O::mul(v0, L[j * ld + c]);
                for (int i = 0; i < m; ++i) d = O::fma(d, A[i * lda + j], A[i * lda + c]);
                const S f = O::mul(d, tau);
                L[j * ld + c] = O::sub(O::mul(f, v0), L[j * ld + c]);
                for (int i = 0; i < m; ++i) A[i * lda + c] = O::sub(A[i * lda + c], O::mul(f, A[i * lda + j]));
            }
            __syncwarp();
            if (lane == 0) L[j * ld + j] = alpha;
        }
        __syncwarp();
    }
}

// Cyclic Jacobi on the symmetric M (R×R, shared), accumulating the rotations
// into E2 (set to I here).  Classic update: M_pp −= t·M_pq, M_qq += t·M_pq,
// M_pq = 0, other entries of rows/columns p, q rotated by (c, s).  Stops when
// every |M_pq| <= tol·sqrt(M_pp·M_qq) or after max_sweeps.  Returns sweeps.
template <class S>
__device__ int warp_jacobi_rel(S *M, S *E2, int R, int ld, float tol, int max_sweeps) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < R * R; i += 32) E2[(i / R) * ld + (i % R)] = (i / R == i % R) ? O::one() : O::zero();
    __syncwarp();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < R - 1; ++p) {
            for (int q = p + 1; q < R; ++q) {
                const S mpq = M[p * ld + q];
                const S mpp = M[p * ld + p];
                const S mqq = M[q * ld + q];
                const float fpq = O::hi(mpq), fpp = O::hi(mpp), fqq = O::hi(mqq);
                __syncwarp();
                if (!(fabsf(fpq) > tol * sqrtf(fabsf(fpp)) * sqrtf(fabsf(fqq)))) continue;
                // the angle only has to be close: approximate reciprocal and
                // square root (the pair (c, s) below is exactly orthogonal)
                const float th = (fqq - fpp) * __frcp_rn(2.0f * fpq);
                float t;
                if (fabsf(th) > 1e18f) t = 0.5f * __frcp_rn(th);
                else {
                    const float h = fmaf(th, th, 1.0f);
                    t = copysignf(__frcp_rn(fabsf(th) + h * rsqrtf(h)), th);
                }
                const S tt = O::from_f(t);
                const S c = O::rsqrt_(O::fma(O::one(), tt, tt));
                const S s = O::mulf(c, t);
                for (int k = lane; k < R; k += 32) {
                    if (k != p && k != q) {
                        const S a = M[p * ld + k], b = M[q * ld + k];
                        const S na = O::sub(O::mul(c, a), O::mul(s, b));
                        const S nb = O::add(O::mul(s, a), O::mul(c, b));
                        M[p * ld + k] = na; M[k * ld + p] = na;
                        M[q * ld + k] = nb; M[k * ld + q] = nb;
                    }
                    const S ea = E2[k * ld + p], eb = E2[k * ld + q];
                    E2[k * ld + p] = O::sub(O::mul(c, ea), O::mul(s, eb));
                    E2[k * ld + q] = O::add(O::mul(s, ea), O::mul(c, eb));
                }
                if (lane == 0) {
                    const S d = O::mulf(mpq, t);
                    M[p * ld + p] = O::sub(mpp, d);
                    M[q * ld + q] = O::add(mqq, d);
                    M[p * ld + q] = O::zero();
                    M[q * ld + p] = O::zero();
                }
                __syncwarp();
                rotated = 1;
            }
        }
        if (!rotated) break;
    }
    __syncwarp();
    return sweep;
}

// Eigen-decomposition of B = LᵀL from its factor: L is R×R upper-triangular
// (shared).  E: on entry an orthogonal basis estimate (I for a cold start),
// on exit the eigenbasis; mu (length R) receives the eigenvalues.  G and M:
// R×ld shared workspaces (G also holds the pass's rotations).  Each pass
// forms G = L·E and M = GᵀG, runs Jacobi on M, then E ← E·(rotations).
// Passes repeat until the freshly formed M starts within omega_stop of
// diagonal (max |M_pq|/sqrt(M_pp M_qq)): Jacobi with FP32 angles and zeroed
// off-diagonals leaves residuals of about 6e-8 times the scaled off-diagonal
// it started from, so the last pass must start nearly diagonal; a cold start
// with cond(B) ~ 1e10 needs 3-4 passes, a warm start 1-2.  Returns the
// passes run.
template <class S>
__device__ int warp_eig_factor(const S *L, S *E, S *G, S *M, S *mu, int R, int ld, int max_passes,
                               float tol, int max_sweeps, float omega_stop) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    int pass = 0;
    while (pass < max_passes) {
        ++pass;
        // G = L E  (row i of L is zero left of the diagonal)
        for (int c = lane; c < R; c += 32)
            for (int i = 0; i < R; ++i) {
                S a = O::zero();
                for (int k = i; k < R; ++k) a = O::fma(a, L[i * ld + k], E[k * ld + c]);
                G[i * ld + c] = a;
            }
        __syncwarp();
        // M = GᵀG, upper triangle computed and mirrored (exactly symmetric)
        for (int b = lane; b < R; b += 32)
            for (int a2 = 0; a2 <= b; ++a2) {
                S s = O::zero();
                for (int i = 0; i < R; ++i) s = O::fma(s, G[i * ld + a2], G[i * ld + b]);
                M[a2 * ld + b] = s;
                M[b * ld + a2] = s;
            }
        __syncwarp();
        // how far from diagonal this pass starts
        float om = 0.f;
        for (int b = lane; b < R; b += 32) {
            const float sb = sqrtf(fabsf(O::hi(M[b * ld + b])));
            for (int a2 = 0; a2 < b; ++a2) {
                const float d = sqrtf(fabsf(O::hi(M[a2 * ld + a2]))) * sb;
                const float x = fabsf(O::hi(M[a2 * ld + b]));
                if (x > 0.f) om = fmaxf(om, d > 0.f ? x / d : 1.f);
            }
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) om = fmaxf(om, __shfl_xor_sync(0xffffffffu, om, m));
        warp_jacobi_rel(M, G, R, ld, tol, max_sweeps);          // rotations → G
        for (int i = lane; i < R; i += 32) mu[i] = M[i * ld + i];
        __syncwarp();
        // E ← E·G (through M)
        for (int c = lane; c < R; c += 32)
            for (int r = 0; r < R; ++r) {
                S a = O::zero();
                for (int k = 0; k < R; ++k) a = O::fma(a, E[r * ld + k], G[k * ld + c]);
                M[r * ld + c] = a;
            }
        __syncwarp();
        for (int i = lane; i < R * R; i += 32) E[(i / R) * ld + (i % R)] = M[(i / R) * ld + (i % R)];
        __syncwarp();
        if (om <= omega_stop) break;
    }
    return pass;
}

template <class A, class B> __device__ __forceinline__ B rt_cast(A a) {
    if constexpr (std::is_same<A, B>::value) return a;
    else return RT<B>::from_d(RT<A>::to_d(a));
}
template <> __device__ __forceinline__ float rt_cast<df, float>(df a) { return a.hi + a.lo; }
template <> __device__ __forceinline__ df rt_cast<float, df>(float a) { return {a, 0.f}; }

// A cheap first pass for warp_eig_factor: the same Gram-Jacobi pass in FP32
// on FP32 copies of L and E (scratch Lf, Ef, Gf, Mf: R×ld floats; muf: R),
// then the refined basis back in S, re-orthogonalised to S precision by two
// Newton–Schulz steps E ← E (3I − EᵀE)/2 (the thousands of FP32 rotations
// leave EᵀE − I near 1e-5; each step squares that).  Gs, Ms: R×ld S
// scratch.  The S passes that follow then start close to diagonal.
template <class S>
__device__ void warp_eig_prepass_f32(const S *L, S *E, float *Lf, float *Ef, float *Gf, float *Mf,
                                     float *muf, S *Gs, S *Ms, int R, int ld, int max_sweeps) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < R * R; i += 32) {
        const int r = i / R, c = i % R;
        Lf[r * ld + c] = rt_cast<S, float>(L[r * ld + c]);
        Ef[r * ld + c] = rt_cast<S, float>(E[r * ld + c]);
    }
    __syncwarp();
    warp_eig_factor<float>(Lf, Ef, Gf, Mf, muf, R, ld, 1, 1e-6f, max_sweeps, 0.f);
    for (int i = lane; i < R * R; i += 32) {
        const int r = i / R, c = i % R;
        E[r * ld + c] = rt_cast<float, S>(Ef[r * ld + c]);
    }
    __syncwarp();
    // twice: P = EᵀE (→ Gs), then E·(3I − P)/2 (→ Ms), copied back to E
    for (int step = 0; step < 2; ++step) {
    for (int b = lane; b < R; b += 32)
        for (int a = 0; a < R; ++a) {
            S acc = O::zero();
            for (int i = 0; i < R; ++i) acc = O::fma(acc, E[i * ld + a], E[i * ld + b]);
            Gs[a * ld + b] = acc;
        }
    __syncwarp();
    for (int c = lane; c < R; c += 32)
        for (int r = 0; r < R; ++r) {
            S acc = O::zero();
            for (int k = 0; k < R; ++k) {
                const S pk = (k == c) ? O::sub(O::from_f(3.f), Gs[k * ld + c]) : O::sub(O::zero(), Gs[k * ld + c]);
                acc = O::fma(acc, E[r * ld + k], pk);
            }
            Ms[r * ld + c] = O::mulf(acc, 0.5f);
        }
    __syncwarp();
    for (int i = lane; i < R * R; i += 32) E[(i / R) * ld + (i % R)] = Ms[(i / R) * ld + (i % R)];
    __syncwarp();
    }
}

// Newton–Schulz steps E ← E (3I − EᵀE)/2 re-orthogonalise E (each step
// squares EᵀE − I: from the few 1e-6 FP32 sweeps leave, one step reaches
// about 1e-11, two the precision of S).  Gs, Ms: R×ld S scratch.
template <class S>
__device__ void warp_newton_schulz(S *E, S *Gs, S *Ms, int R, int ld, int steps) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    for (int step = 0; step < steps; ++step) {
        for (int b = lane; b < R; b += 32)
            for (int a = 0; a < R; ++a) {
                S acc = O::zero();
                for (int i = 0; i < R; ++i) acc = O::fma(acc, E[i * ld + a], E[i * ld + b]);
                Gs[a * ld + b] = acc;
            }
        __syncwarp();
        for (int c = lane; c < R; c += 32)
            for (int r = 0; r < R; ++r) {
                S acc = O::zero();
                for (int k = 0; k < R; ++k) {
                    const S pk = (k == c) ? O::sub(O::from_f(3.f), Gs[k * ld + c]) : O::sub(O::zero(), Gs[k * ld + c]);
                    acc = O::fma(acc, E[r * ld + k], pk);
                }
                Ms[r * ld + c] = O::mulf(acc, 0.5f);
            }
        __syncwarp();
        for (int i = lane; i < R * R; i += 32) E[(i / R) * ld + (i % R)] = Ms[(i / R) * ld + (i % R)];
        __syncwarp();
    }
}

// warp_newton_schulz for R <= 32 with one shared scratch block: lane c holds
// column c of P = EᵀE in registers, writes column c of E (3I − P)/2 to Es,
// and Es is copied back to E.  The same arithmetic as warp_newton_schulz.
template <class S>
__device__ void warp_newton_schulz_reg(S *E, S *Es, int R, int ld, int steps) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    const bool act = lane < R;
    for (int step = 0; step < steps; ++step) {
        S p[32];
#pragma unroll
        for (int a = 0; a < 32; ++a) {
            S acc = O::zero();
            if (act && a < R)
                for (int i = 0; i < R; ++i) acc = O::fma(acc, E[i * ld + a], E[i * ld + lane]);
            p[a] = acc;
        }
        if (act)
            for (int r = 0; r < R; ++r) {
                S acc = O::zero();
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k < R) {
                        const S pk = (k == lane) ? O::sub(O::from_f(3.f), p[k]) : O::sub(O::zero(), p[k]);
                        acc = O::fma(acc, E[r * ld + k], pk);
                    }
                Es[r * ld + lane] = O::mulf(acc, 0.5f);
            }
        __syncwarp();
        for (int i = lane; i < R * R; i += 32) E[(i / R) * ld + (i % R)] = Es[(i / R) * ld + (i % R)];
        __syncwarp();
    }
}

// One-sided (Hestenes) Jacobi for the eigen-decomposition of B = LᵀL, R <= 32,
// register-resident: lane c holds column c of G = L·E and of E in the
// working type W (S, or float for a cheap first pass).  A sweep pairs every
// column with every other once: in round m (1..31) lane c meets lane c^m
// (a perfect matching; pair (i, j) meets in round i^j), and each pair is
// rotated so that its two columns of G become orthogonal: with α = |g_i|²,
// β = |g_j|², γ = g_i·g_j (i < j), θ = (β − α)/(2γ),
// t = sign(θ)/(|θ| + sqrt(1 + θ²)), c = 1/sqrt(1 + t²), s = c·t,
// g_i ← c g_i − s g_j, g_j ← s g_i + c g_j, and the same on E's columns.
// The lower lane of the pair computes t (in FP32: the angle need only be
// close, the pair (c, s) in W is exactly orthogonal) and passes it to its
// partner, so both apply one rotation.  Sweeps stop when every
// |γ| <= tol·sqrt(αβ) or after max_sweeps, or (stop > 0) after a sweep whose
// largest rotated cosine was <= stop: cyclic Jacobi converges quadratically
// near the end, so a sweep that starts at cosines δ leaves O(δ²), below tol
// when stop <= sqrt(tol)/2, and the confirming sweep is skipped.  On exit the columns of G are
// orthogonal: E (smem, S) holds the eigenvectors and mu[c] = |g_c|² (S)
// the eigenvalues.  Rotating G itself, never forming LᵀL, keeps the
// relative accuracy of one-sided Jacobi (Demmel and Veselić 1992).  L (smem,
// S, upper triangular) is read only.  Returns the sweeps run.
template <class W, class S>
__device__ int warp_eig_os(const S *L, S *E, S *mu, int R, int ld, int max_sweeps, float tol,
                            float stop = 0.f) {
    using O = RT<W>;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool act = lane < R;
    W g[32], e[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) e[i] = (act && i < R) ? rt_cast<S, W>(E[i * ld + lane]) : O::zero();
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        W a = O::zero();
        if (i < R)
#pragma unroll
            for (int k = i; k < 32; ++k)
                if (k < R) a = O::fma(a, rt_cast<S, W>(L[i * ld + k]), e[k]);
        g[i] = a;
    }
    // Columns whose squared norm is below tol²·‖L‖_F² count as zero and are not
    // rotated: in a rank-deficient L such a column stays collinear with a
    // large one, so the cosine test alone would keep rotating it until it
    // underflows (and a denormal γ would turn θ into 0·∞).
    float fro = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) fro = fmaf(O::hi(g[i]), O::hi(g[i]), fro);
#pragma unroll
    for (int o = 16; o; o >>= 1) fro += __shfl_xor_sync(full, fro, o);
    const float flo = tol * tol * fro;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        float off = 0.f;
        for (int m = 1; m < 32; ++m) {
            const int p = lane ^ m;
            // γ in the working type, in two interleaved chains (ILP); the
            // norms only steer the angle and the skip tests, which run in
            // FP32, so they are summed in FP32 from the leading parts
            W dot0 = O::zero(), dot1 = O::zero();
            float nnf = 0.f;
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                const W gp0 = O::shfl_xor(g[i], m);
                const W gp1 = O::shfl_xor(g[i + 1], m);
                dot0 = O::fma(dot0, g[i], gp0);
                dot1 = O::fma(dot1, g[i + 1], gp1);
                nnf = fmaf(O::hi(g[i]), O::hi(g[i]), nnf);
                nnf = fmaf(O::hi(g[i + 1]), O::hi(g[i + 1]), nnf);
            }
            const W dot = O::add(dot0, dot1);
            const float np = __shfl_xor_sync(full, nnf, m);
            const bool lo = lane < p;
            float t = 0.f;
            const float al = nnf, be = np;
            if (lo && act && p < R && al > flo && be > flo) {   // this lane is i, the partner j
                const float ga = O::hi(dot);
                const float sc = sqrtf(al) * sqrtf(be);
                if (fabsf(ga) > tol * sc) {
                    off = fmaxf(off, fabsf(ga) / sc);
                    const float df = be - al;
                    const float th = df == 0.f ? 0.f : df * __frcp_rn(2.0f * ga);
                    if (fabsf(th) > 1e18f) t = 0.5f * __frcp_rn(th);
                    else {
                        const float h = fmaf(th, th, 1.0f);
                        t = copysignf(__frcp_rn(fabsf(th) + h * rsqrtf(h)), th);
                    }
                }
            }
            const float tp = __shfl_xor_sync(full, t, m);
            t = lo ? t : tp;
            if (__any_sync(full, t != 0.f)) {
                const W tt = O::from_f(t);
                const W c = O::rsqrt_(O::fma(O::one(), tt, tt));
                const W sg = O::mulf(c, lo ? -t : t);     // i: c g_i − s g_j; j: c g_j + s g_i
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const W gp = O::shfl_xor(g[i], m);
                    g[i] = O::fma(O::mul(c, g[i]), sg, gp);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const W ep = O::shfl_xor(e[i], m);
                    e[i] = O::fma(O::mul(c, e[i]), sg, ep);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) off = fmaxf(off, __shfl_xor_sync(full, off, o));
        if (off <= stop) {
            ++sweep;
            break;
        }
    }
    W nn = O::zero();
#pragma unroll
    for (int i = 0; i < 32; ++i) nn = O::fma(nn, g[i], g[i]);
    __syncwarp();
    if (act) {
        if (mu) mu[lane] = rt_cast<W, S>(nn);
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i < R) E[i * ld + lane] = rt_cast<W, S>(e[i]);
    }
    __syncwarp();
    return sweep;
}

// Spectral weights of B^{-1/2} and B^{1/2} from the eigenvalues mu:
// finv_i = μ_i^{-1/2} and fsq_i = μ_i^{1/2} for μ_i > rtol·max μ, both 0
// otherwise (the pseudo-inverse cut; B^{1/2}·B^{-1/2} is then the projector
// on the kept eigenvectors).
template <class S>
__device__ void warp_sqrt_weights(const S *mu, int R, double rtol, S *finv, S *fsq) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int i = lane; i < R; i += 32) mx = fmax(mx, O::to_d(mu[i]));
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, m));
    for (int i = lane; i < R; i += 32) {
        const S v = mu[i];
        const bool keep = mx > 0.0 && O::to_d(v) > rtol * mx;
        finv[i] = keep ? O::rsqrt_(v) : O::zero();
        fsq[i] = keep ? O::sqrt_(v) : O::zero();
    }
    __syncwarp();
}

// out = E diag(f) Eᵀ (R×R, shared, ld), out must not alias E.
template <class S>
__device__ void warp_spectral_s(const S *E, const S *f, int R, int ld, S *out) {
    using O = RT<S>;
    const int lane = threadIdx.x & 31;
    for (int idx = lane; idx < R * R; idx += 32) {
        const int r = idx / R, c = idx % R;
        S a = O::zero();
        for (int k = 0; k < R; ++k) a = O::fma(a, O::mul(E[r * ld + k], f[k]), E[c * ld + k]);
        out[r * ld + c] = a;
    }
    __syncwarp();
}

}  // namespace dash
