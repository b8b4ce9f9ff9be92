// k_seq.cu -- the deflation term of Alg. 3 (sequential ALS, Sec. 4).  With
// the converged topics U1 (n x k1) and V1 (m x k1) held densely, the updates
// of the new block U2 (n x k2), V2 (m x k2) are
//   V2 = (A^T U2 - V1 (U1^T U2)) (U2^T U2)^-1      (Eq. 7)
//   U2 = (A V2 - U1 (V1^T V2)) (V2^T V2)^-1        (Eq. 8)
// The sparse product A^T U2 (A V2), the k2 x k2 Gram solve, the projection
// and the top-t rule are those of Alg. 2 with k = k2; these kernels supply
// the term in between: g = G1^T F (k1 x k2: the converged topics of the
// factor that is held fixed against its new block F) and Y -= H1 g (the
// converged topics of the factor being updated).  Sums in FP64, in a fixed
// order.
#include "common.cuh"

namespace espnmf {

constexpr int kSeqThreads = 256;

// g[c * k2 + j] = sum_i G1[i][c] F[i][j] for c < k1, j < k2 (one block per
// (c, j); the grid covers the largest k1, *k1 is read on the device so that
// one captured sweep serves every block of topics), over the rows where F --
// row-packed: cnt[i] pairs (column, value) at [i * ld, i * ld + cnt[i]) --
// has column j.  Per-thread sums in row order, then a fixed tree.
template <typename T>
__global__ void __launch_bounds__(kSeqThreads)
seq_dot_kernel(int64_t rows, const T* __restrict__ G1, int ld1, const int32_t* __restrict__ cnt,
               const int32_t* __restrict__ col, const T* __restrict__ val, int ld, int k2,
               const int* __restrict__ k1p, double* __restrict__ g)
{
    __shared__ double red[kSeqThreads];
    const int c = blockIdx.x, j = blockIdx.y;
    if (c >= *k1p) return;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += kSeqThreads) {
        const int nc = cnt[i];
        for (int q = 0; q < nc; ++q)
            if (col[i * ld + q] == j) {
                s = fma((double)G1[i * ld1 + c], (double)val[i * ld + q], s);
                break;
            }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = kSeqThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[c * k2 + j] = red[0];
}

// Y[i][j] -= sum_{c < k1} H1[i][c] g[c][j], one thread per row (row stride
// ldy); the sum is formed in FP64 in c order (zero entries of H1 add
// nothing and are skipped) and the difference rounded once.
template <typename T>
__global__ void __launch_bounds__(kSeqThreads)
seq_deflate_kernel(int64_t rows, const int* __restrict__ k1p, int k2, const T* __restrict__ H1,
                   int ld1, const double* __restrict__ g, T* __restrict__ Y, int64_t ldy)
{
    const int64_t i = (int64_t)blockIdx.x * kSeqThreads + threadIdx.x;
    const int k1 = *k1p;
    if (i >= rows || k1 <= 0) return;
    const T* h = H1 + i * ld1;
    for (int j = 0; j < k2; ++j) {
        double s = 0.0;
        for (int c = 0; c < k1; ++c) {
            const double hc = (double)h[c];
            if (hc != 0.0) s = fma(hc, g[c * k2 + j], s);
        }
        Y[i * ldy + j] = (T)((double)Y[i * ldy + j] - s);
    }
}

// H[i][j0 + j] = the block factor's value in row i, column j (0 where it
// has none), for j < k2.
template <typename T>
__global__ void __launch_bounds__(kSeqThreads)
seq_append_kernel(int64_t rows, const int32_t* __restrict__ cnt, const int32_t* __restrict__ col,
                  const T* __restrict__ val, int ld, int k2, T* __restrict__ H, int ld1, int j0)
{
    const int64_t i = (int64_t)blockIdx.x * kSeqThreads + threadIdx.x;
    if (i >= rows) return;
    T* h = H + i * ld1 + j0;
    for (int j = 0; j < k2; ++j) h[j] = T(0);
    const int nc = cnt[i];
    for (int q = 0; q < nc; ++q) {
        const int c = col[i * ld + q];
        if (ESPNMF_CHECK((unsigned)c < (unsigned)k2, CHK_COLUMN)) h[c] = val[i * ld + q];
    }
}

ESPNMF_CHECK_READER(check_flags_seq)

static unsigned seq_grid(int64_t rows) { return (unsigned)((rows + kSeqThreads - 1) / kSeqThreads); }

template <typename T>
cudaError_t launch_seq_deflate(int64_t rows_f, const T* G1, int64_t rows_h, const T* H1, int ld1,
                               int k1_max, const int* k1, int k2, const int32_t* cnt,
                               const int32_t* col, const T* val, int ld, double* g, T* Y,
                               int64_t ldy, cudaStream_t st)
{
    if (k1_max <= 0) return cudaSuccess;
    seq_dot_kernel<T><<<dim3((unsigned)k1_max, (unsigned)k2), kSeqThreads, 0, st>>>(
        rows_f, G1, ld1, cnt, col, val, ld, k2, k1, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || rows_h == 0) return e;
    seq_deflate_kernel<T><<<seq_grid(rows_h), kSeqThreads, 0, st>>>(rows_h, k1, k2, H1, ld1, g, Y, ldy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_seq_append(int64_t rows, const int32_t* cnt, const int32_t* col, const T* val,
                              int ld, int k2, T* H, int ld1, int j0, cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    seq_append_kernel<T><<<seq_grid(rows), kSeqThreads, 0, st>>>(rows, cnt, col, val, ld, k2, H, ld1, j0);
    return cudaGetLastError();
}

template cudaError_t launch_seq_deflate<float>(int64_t, const float*, int64_t, const float*, int, int,
                                               const int*, int, const int32_t*, const int32_t*,
                                               const float*, int, double*, float*, int64_t,
                                               cudaStream_t);
template cudaError_t launch_seq_deflate<double>(int64_t, const double*, int64_t, const double*, int,
                                                int, const int*, int, const int32_t*, const int32_t*,
                                                const double*, int, double*, double*, int64_t,
                                                cudaStream_t);
template cudaError_t launch_seq_append<float>(int64_t, const int32_t*, const int32_t*, const float*,
                                              int, int, float*, int, int, cudaStream_t);
template cudaError_t launch_seq_append<double>(int64_t, const int32_t*, const int32_t*,
                                               const double*, int, int, double*, int, int,
                                               cudaStream_t);

}  // namespace espnmf
