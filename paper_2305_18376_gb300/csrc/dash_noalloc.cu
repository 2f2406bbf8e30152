// Allocation-free F increment: F_inc = Σ_k X_k,newᵀ U_k,new S_k, the new-data
// term that dash_update() adds to λF (Eq. 20), for callers that may not
// allocate device memory themselves or let a library do it.
//
// Who needs it: code that runs inside a host framework whose memory manager
// owns the whole device and forbids outside cudaMalloc; latency-bound serving
// loops, where a cudaMalloc/cudaFree can synchronise the device and stall work
// already in flight; and processes that must fix their device footprint at
// start-up.  Such a caller passes its own inputs and output; the per-block
// partial sums live in g_noalloc_partials below instead of a cudaMalloc'd
// buffer.
//
// The partial-sum array is a file-scope __device__ array of
// kNoallocPartialFloats floats (8 MiB).  Every GPU that loads this library
// holds it until the process exits.  All calls share it: two calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race on it and must be serialised by the caller.  Each call writes
// every partial slot it later reads, so nothing has to start at zero and the
// contents a previous call left behind are never read.
//
// In host code the symbol g_noalloc_partials is only a host-side stand-in for
// the array, not its device address, so the address is looked up with
// cudaGetSymbolAddress (with the device current).  A call on a stream that is
// not being captured looks it up afresh and caches it per device, so a
// context torn down and created again (cudaDeviceReset) is picked up; a call
// made while its stream is being captured into a CUDA graph uses the cached
// address, so the first call on each device must come before any capture.
#include <cuda_runtime.h>

#include <mutex>

#include "dash.h"

namespace {

constexpr int64_t kNoallocPartialFloats = int64_t(1) << 21;   // 8 MiB of FP32 partials
constexpr int kNoallocChunksMax = 64;                          // row chunks (partials) per call
constexpr int kJB = 64;                                        // columns per CTA
constexpr int kRC = 32;                                        // rows staged per pass
constexpr int kRMax = 64;

__device__ __align__(256) float g_noalloc_partials[kNoallocPartialFloats];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
float *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device: looked up when
// `stream` is not being captured (and cached), the cached one during capture.
cudaError_t partials_address(cudaStream_t stream, float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<float *>(p);
    } else if (!g_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;   // first call on this device is under capture
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Partials of Σ_rows X(i,:)ᵀ (U(i,:) ∘ W(k(i),:)) for one row chunk (blockIdx.x)
// and 64 columns (blockIdx.y); k(i) is found by binary search in seg_row.
__global__ void __launch_bounds__(256) k_f_noalloc(const float *__restrict__ X,
                                                   const float *__restrict__ U, int64_t N, int J,
                                                   int R, const int64_t *__restrict__ seg_row,
                                                   const int *__restrict__ seg_slice, int n_seg,
                                                   const double *__restrict__ W,
                                                   int64_t rows_per_chunk,
                                                   float *__restrict__ partials) {
    __shared__ float Xs[kRC][kJB + 1];
    __shared__ float Us[kRC][kRMax];
    __shared__ int ks[kRC];
    const int tid = threadIdx.x;
    const int jj = tid % kJB, rg = tid / kJB;
    const int j0 = blockIdx.y * kJB;
    const int64_t rbeg = (int64_t)blockIdx.x * rows_per_chunk;
    const int64_t rend = (N < rbeg + rows_per_chunk) ? N : rbeg + rows_per_chunk;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    for (int64_t c0 = rbeg; c0 < rend; c0 += kRC) {
        const int nr = (int)((rend - c0) < kRC ? (rend - c0) : kRC);
        __syncthreads();
        if (tid < nr) {
            const int64_t i = c0 + tid;
            int lo = 0, hi = n_seg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_row[mid] <= i) lo = mid; else hi = mid - 1;
            }
            while (lo + 1 < n_seg && seg_row[lo + 1] <= i) ++lo;
            ks[tid] = seg_slice[lo];
        }
        for (int e = tid; e < kRC * kJB; e += 256) {
            const int i = e / kJB, j = e % kJB;
            Xs[i][j] = (i < nr && j0 + j < J) ? X[(c0 + i) * J + j0 + j] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < kRC * R; e += 256) {
            const int i = e / R, r = e % R;
            Us[i][r] = (i < nr) ? U[(c0 + i) * R + r] * (float)W[(int64_t)ks[i] * R + r] : 0.f;
        }
        __syncthreads();
        for (int i = 0; i < nr; ++i) {
            const float x = Xs[i][jj];
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
            if (r < R) partials[((int64_t)blockIdx.x * J + j0 + jj) * R + r] = acc[q];
        }
    }
}

// F_inc[i] = Σ_b partials[b][i] in a fixed order, FP64.
__global__ void k_f_noalloc_sum(const float *__restrict__ partials, int nb, int64_t JR,
                                double *__restrict__ F_inc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= JR) return;
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += (double)partials[(int64_t)b * JR + i];
    F_inc[i] = a;
}

}  // namespace

extern "C" dash_status dash_f_increment_noalloc(const float *X, const float *U, int64_t N,
                                                int32_t J, int32_t R, const int64_t *seg_row,
                                                const int32_t *seg_slice, int64_t n_seg,
                                                const double *W, double *F_inc, void *stream) {
    if (J <= 0 || R < 1 || R > kRMax || N < 0 || n_seg < 0 || n_seg > INT32_MAX) return DASH_EINVAL;
    if (!F_inc || (N > 0 && (!X || !U || !seg_row || !seg_slice || !W || n_seg == 0)))
        return DASH_EINVAL;
    const int64_t JR = (int64_t)J * R;
    if (JR > kNoallocPartialFloats) return DASH_ENOMEM;      // J·R beyond the static array
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *partials = nullptr;
    if (partials_address(st, &partials) != cudaSuccess) {
        cudaGetLastError();
        return DASH_ECUDA;
    }
    int nb = 0;
    if (N > 0) {
        const int64_t by_size = kNoallocPartialFloats / JR;
        int64_t want = (N + kRC - 1) / kRC;
        if (want > kNoallocChunksMax) want = kNoallocChunksMax;
        if (want > by_size) want = by_size;
        int64_t rpc = (N + want - 1) / want;
        rpc = (rpc + kRC - 1) / kRC * kRC;
        nb = (int)((N + rpc - 1) / rpc);
        dim3 grid(nb, (J + kJB - 1) / kJB);
        k_f_noalloc<<<grid, 256, 0, st>>>(X, U, N, J, R, seg_row, seg_slice, (int)n_seg, W, rpc,
                                          partials);
        if (cudaGetLastError() != cudaSuccess) return DASH_ECUDA;
    }
    k_f_noalloc_sum<<<(int)((JR + 255) / 256), 256, 0, st>>>(partials, nb, JR, F_inc);
    if (cudaGetLastError() != cudaSuccess) return DASH_ECUDA;
    return DASH_OK;
}
