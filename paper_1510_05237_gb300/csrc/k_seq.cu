// k_seq.cu -- the deflation term of Alg. 3 (sequential ALS, Sec. 4) for a
// rank-1 new topic (k2 = 1).  With the converged topics U1 (n x k1) and V1
// (m x k1) held densely, the updates of the new topic u, v are
//   v = (A^T u - V1 (U1^T u)) / (u^T u)      (Eq. 7)
//   u = (A v - U1 (V1^T v)) / (v^T v)        (Eq. 8)
// The sparse product A^T u (A v), the division by the 1 x 1 Gram, the
// projection and the top-t rule are those of Alg. 2 with k = 1; these
// kernels supply the term in between: g = G1^T f (the converged topics of
// the factor that is held fixed against its new column f) and Y -= H1 g
// (the converged topics of the factor being updated).  Sums in FP64, in a
// fixed order.
#include "common.cuh"

namespace espnmf {

constexpr int kSeqThreads = 256;

// g[c] = sum_i G1[i][c] f_i for c < k1 (one block per c), over the rows
// where the rank-1 factor f -- row-packed: cnt[i] in {0, 1}, value
// val[i * ld] -- is nonzero.  Per-thread sums in row order, then a fixed
// tree.
template <typename T>
__global__ void __launch_bounds__(kSeqThreads)
seq_dot_kernel(int64_t rows, const T* __restrict__ G1, int ld1, const int32_t* __restrict__ cnt,
               const T* __restrict__ val, int ld, double* __restrict__ g)
{
    __shared__ double red[kSeqThreads];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += kSeqThreads)
        if (cnt[i] > 0) s = fma((double)G1[i * ld1 + c], (double)val[i * ld], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = kSeqThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[c] = red[0];
}

// Y[i] -= sum_{c < k1} H1[i][c] g[c], one thread per row (column 0 of Y,
// row stride ldy); the difference is formed in FP64 and rounded once.
template <typename T>
__global__ void __launch_bounds__(kSeqThreads)
seq_deflate_kernel(int64_t rows, int k1, const T* __restrict__ H1, int ld1,
                   const double* __restrict__ g, T* __restrict__ Y, int64_t ldy)
{
    const int64_t i = (int64_t)blockIdx.x * kSeqThreads + threadIdx.x;
    if (i >= rows) return;
    double s = 0.0;
    for (int c = 0; c < k1; ++c) s = fma((double)H1[i * ld1 + c], g[c], s);
    Y[i * ldy] = (T)((double)Y[i * ldy] - s);
}

// H[i][j] = the rank-1 factor's value in row i (0 where it has none).
template <typename T>
__global__ void __launch_bounds__(kSeqThreads)
seq_append_kernel(int64_t rows, const int32_t* __restrict__ cnt, const T* __restrict__ val, int ld,
                  T* __restrict__ H, int ld1, int j)
{
    const int64_t i = (int64_t)blockIdx.x * kSeqThreads + threadIdx.x;
    if (i >= rows) return;
    H[i * ld1 + j] = cnt[i] > 0 ? val[i * ld] : T(0);
}

static unsigned seq_grid(int64_t rows) { return (unsigned)((rows + kSeqThreads - 1) / kSeqThreads); }

template <typename T>
cudaError_t launch_seq_deflate(int64_t rows_f, const T* G1, int64_t rows_h, const T* H1, int ld1,
                               int k1, const int32_t* cnt, const T* val, int ld, double* g, T* Y,
                               int64_t ldy, cudaStream_t st)
{
    if (k1 <= 0) return cudaSuccess;
    seq_dot_kernel<T><<<(unsigned)k1, kSeqThreads, 0, st>>>(rows_f, G1, ld1, cnt, val, ld, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || rows_h == 0) return e;
    seq_deflate_kernel<T><<<seq_grid(rows_h), kSeqThreads, 0, st>>>(rows_h, k1, H1, ld1, g, Y, ldy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_seq_append(int64_t rows, const int32_t* cnt, const T* val, int ld, T* H, int ld1,
                              int j, cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    seq_append_kernel<T><<<seq_grid(rows), kSeqThreads, 0, st>>>(rows, cnt, val, ld, H, ld1, j);
    return cudaGetLastError();
}

template cudaError_t launch_seq_deflate<float>(int64_t, const float*, int64_t, const float*, int, int,
                                               const int32_t*, const float*, int, double*, float*,
                                               int64_t, cudaStream_t);
template cudaError_t launch_seq_deflate<double>(int64_t, const double*, int64_t, const double*, int,
                                                int, const int32_t*, const double*, int, double*,
                                                double*, int64_t, cudaStream_t);
template cudaError_t launch_seq_append<float>(int64_t, const int32_t*, const float*, int, float*, int,
                                              int, cudaStream_t);
template cudaError_t launch_seq_append<double>(int64_t, const int32_t*, const double*, int, double*,
                                               int, int, cudaStream_t);

}  // namespace espnmf
