// k_metrics.cu -- the document-clustering accuracy of a topic model (Sec.
// 3.2, Eq. 3 and 4) from a factor on the device.
//
// Document i belongs to topic c when entry (i, c) of the factor is nonzero.
// For topic c with n_D members from n_J classes, P = sum_j h_j (h_j - 1) / 2
// (h_j: members of class j) counts the member pairs that share a class,
// alpha = q (n_J (q - 1) / 2 + r) with q = n_D div n_J, r = n_D mod n_J is
// that count for the most even spread of n_D members over the classes, and
// beta = n_D (n_D - 1) / 2 the count of all pairs; Acc = (P - alpha) /
// (beta - alpha), 1 for a topic of at most one member or when beta = alpha.
//
// Pass 1 adds one to hist[c * n_J + label] for every nonzero (i, c) of the
// row-packed factor (integer atomics: the counts do not depend on the
// order); pass 2 forms each column's accuracy in FP64 from its histogram.
#include "common.cuh"

namespace espnmf {

__global__ void class_hist_kernel(int64_t rows, int ld, const int32_t* __restrict__ cnt,
                                  const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ labels, int n_classes,
                                  unsigned* hist, unsigned* status)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int c_n = cnt[r];
        if (c_n == 0) continue;
        const int lab = labels[r];
        if (lab < 0 || lab >= n_classes) {
            atomicOr(status, ST_BADINPUT);
            continue;
        }
        for (int q = 0; q < c_n; ++q)
            atomicAdd(hist + (int64_t)col[r * ld + q] * n_classes + lab, 1u);
    }
}

__global__ void topic_accuracy_kernel(int k, int n_classes, const unsigned* __restrict__ hist,
                                      double* acc)
{
    const int c = blockIdx.x;
    __shared__ double s_pairs[256];
    __shared__ unsigned long long s_n[256];
    double pairs = 0.0;
    unsigned long long nd = 0;
    for (int j = threadIdx.x; j < n_classes; j += blockDim.x) {
        const double h = (double)hist[(int64_t)c * n_classes + j];
        pairs += h * (h - 1.0) / 2.0;
        nd += hist[(int64_t)c * n_classes + j];
    }
    s_pairs[threadIdx.x] = pairs;
    s_n[threadIdx.x] = nd;
    __syncthreads();
    if (threadIdx.x == 0) {
        double P = 0.0;
        unsigned long long n = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {   // fixed order
            P += s_pairs[t];
            n += s_n[t];
        }
        double a = 1.0;
        if (n > 1) {
            const unsigned long long q = n / (unsigned long long)n_classes;
            const unsigned long long r = n % (unsigned long long)n_classes;
            const double alpha = (double)q * ((double)n_classes * ((double)q - 1.0) / 2.0 + (double)r);
            const double beta = (double)n * ((double)n - 1.0) / 2.0;
            if (beta != alpha) a = (P - alpha) / (beta - alpha);
        }
        acc[c] = a;
    }
}

cudaError_t launch_topic_accuracy(const EllDev& F, int k, const int32_t* labels, int n_classes,
                                  unsigned* hist, double* acc, unsigned* status, int sm_count,
                                  cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * (size_t)k * n_classes, st);
    if (e != cudaSuccess) return e;
    if (F.rows > 0) {
        int64_t grid = (F.rows + 255) / 256;
        if (grid > 8 * sm_count) grid = 8 * sm_count;
        class_hist_kernel<<<(unsigned)grid, 256, 0, st>>>(F.rows, F.ld, F.cnt, F.col, labels,
                                                          n_classes, hist, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    topic_accuracy_kernel<<<k, 256, 0, st>>>(k, n_classes, hist, acc);
    return cudaGetLastError();
}

}  // namespace espnmf
