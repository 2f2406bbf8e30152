// Reconstruction errors of an update's new data (Definitions 1-2, the
// slice-level and tensor-level reconstruction errors): a second read of
// X_new against X̂_new = U_k,new S_k Vᵀ (mode P) or Q_k,new H S_k Vᵀ (mode Q)
// with the updated factors.
//
//   k_resid_rows   one warp per row: Σ_j |x − x̂|, Σ_j (x − x̂)², Σ_j x²  (FP64)
//   k_resid_segs   one thread per segment: the three sums over its rows, in
//                  row order (the host groups segments by slice)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dash_kernels_p.cuh"

namespace dash {

template <typename T>
__host__ __device__ inline int err_chunk(int R, int J) {
    const int Jp = ((J + 127) / 128) * 128;
    int cap = (int)((180 * 1024) / ((size_t)R * sizeof(T)) / 128) * 128;
    if (cap < 128) cap = 128;
    return Jp < cap ? Jp : cap;
}
template <typename T>
__host__ __device__ inline size_t err_smem(int R, int J) {
    return ((size_t)R * err_chunk<T>(R, J) + 8 * 64) * sizeof(T);
}

// rows: N×R new factor rows (U for mode P, Q for mode Q); H: R×R (mode Q)
// or null (mode P); W, V: the updated factors (V in the product type).
template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_resid_rows(int64_t N, int J, int R, int n_seg,
                                                    const int64_t *__restrict__ seg_row,
                                                    const int *__restrict__ seg_slice,
                                                    const TI *__restrict__ X, const T *__restrict__ rows,
                                                    const double *__restrict__ H,
                                                    const double *__restrict__ W,
                                                    const T *__restrict__ VT,
                                                    double *__restrict__ out /* N×3 */) {
    extern __shared__ unsigned char er_raw[];
    const int Jc = err_chunk<T>(R, J);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *Vt = reinterpret_cast<T *>(er_raw);                    // R × Jc
    T *zs = Vt + (size_t)R * Jc + (size_t)wid * 64;
    for (int jb = 0; jb < J; jb += Jc) {
        __syncthreads();
        for (int e = threadIdx.x; e < R * Jc; e += blockDim.x) {
            const int s2 = e / Jc, j = jb + e % Jc;
            Vt[e] = j < J ? VT[(int64_t)j * R + s2] : T(0);
        }
        __syncthreads();
        for (int64_t row = (int64_t)blockIdx.x * nw + wid; row < N; row += (int64_t)gridDim.x * nw) {
            // slice of this row: last segment starting at or before it
            int lo = 0, hi = n_seg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_row[mid] <= row) lo = mid; else hi = mid - 1;
            }
            while (lo + 1 < n_seg && seg_row[lo + 1] <= row) ++lo;
            const int k = seg_slice[lo];
            __syncwarp();
            for (int s2 = lane; s2 < R; s2 += 32) {
                T a;
                if (H) {
                    a = T(0);
                    for (int r = 0; r < R; ++r) a += rows[row * R + r] * (T)H[r * R + s2];
                } else {
                    a = rows[row * R + s2];
                }
                zs[s2] = a * (T)W[(int64_t)k * R + s2];
            }
            __syncwarp();
            double sa = 0.0, sq = 0.0, sx = 0.0;
            const TI *xr = X + row * J + jb;
            for (int j0 = 4 * lane; j0 < Jc && jb + j0 < J; j0 += 128) {
                T h[4] = {T(0), T(0), T(0), T(0)};
                for (int s2 = 0; s2 < R; ++s2) {
                    const T z = zs[s2];
                    const T *v = Vt + (size_t)s2 * Jc + j0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) h[u] += z * v[u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jb + j0 + u < J) {
                        const double x = (double)xr[j0 + u];
                        const double d = x - (double)h[u];
                        sa += fabs(d);
                        sq += d * d;
                        sx += x * x;
                    }
                }
            }
            sa = warp_sum(sa);
            sq = warp_sum(sq);
            sx = warp_sum(sx);
            if (lane == 0) {
                double *o = out + row * 3;
                if (jb == 0) { o[0] = sa; o[1] = sq; o[2] = sx; }
                else { o[0] += sa; o[1] += sq; o[2] += sx; }
            }
        }
    }
}

static __global__ void k_resid_segs(int n_seg, const int64_t *__restrict__ seg_row,
                             const double *__restrict__ rowsum, double *__restrict__ segsum) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seg) return;
    double a = 0.0, q = 0.0, x = 0.0;
    for (int64_t r = seg_row[s]; r < seg_row[s + 1]; ++r) {
        a += rowsum[r * 3];
        q += rowsum[r * 3 + 1];
        x += rowsum[r * 3 + 2];
    }
    segsum[s * 3] = a;
    segsum[s * 3 + 1] = q;
    segsum[s * 3 + 2] = x;
}

}  // namespace dash
