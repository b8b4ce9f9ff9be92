// k_grad.cu -- the differentiable-loss helpers around the squared objective
// (Eq. 6), f(U, V) = ||A - U V^T||_F^2:
//
//   grad          dense gradient of f with respect to one factor F (U or V),
//                   grad_F = 2 (F G_O - Y),   G_O = O^T O,  Y = A V or A^T U,
//                 from F's row-packed nonzeros, the FP64 Gram of the other
//                 factor O and the sparse product Y of the current sweep.
//   lambda_max    the largest eigenvalue of G_O by 20 power-iteration steps
//                 from the normalised all-ones vector (FP64, one CTA), for
//                 the Lipschitz step eta = 1 / (2 lambda_max).
//   pg_apply      one projected-gradient step on F's current support S:
//                   F <- P_S(F - eta grad_F),
//                 P_S clamping to >= 0 and keeping only entries in S; the
//                 result is written column-major as a candidate for the
//                 factor emit (with every positive entry kept).
//
// The F G_O products run in FP64 over F's nonzeros only (at most t per
// column), so their cost is nnz(F) * k FMAs.
#include "common.cuh"

namespace espnmf {

// One thread per output element, row-major (consecutive threads take
// consecutive columns of a row, so the stores and the reads of Y coalesce).
template <typename T, typename OutT>
__global__ void grad_kernel(int64_t rows, int k, EllDev F, const double* __restrict__ Go,
                            const T* __restrict__ Y, int64_t ldy, OutT* __restrict__ out)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rows * k) return;
    const int64_t r = g / k;
    const int c = (int)(g - r * k);
    const int cnt = F.cnt[r];
    const int32_t* col = F.col + r * F.ld;
    const T* val = static_cast<const T*>(F.val) + r * F.ld;
    double s = 0.0;
    for (int q = 0; q < cnt; ++q) s = fma((double)val[q], Go[(int64_t)col[q] * k + c], s);
    out[g] = (OutT)(2.0 * (s - (double)Y[r * ldy + c]));
}

template <typename T, typename OutT>
cudaError_t launch_grad(int64_t rows, int k, const EllDev& F, const double* Go, const T* Y,
                        int64_t ldy, OutT* out, cudaStream_t st)
{
    const int64_t total = rows * k;
    if (total == 0) return cudaSuccess;
    const int B = 256;
    grad_kernel<T, OutT><<<(unsigned)((total + B - 1) / B), B, 0, st>>>(rows, k, F, Go, Y, ldy, out);
    return cudaGetLastError();
}

// Power iteration in the order of its definition: y = G x (sums over d in
// ascending order), lambda = ||y||_2 (sums over c in ascending order),
// x = y / lambda.  Products and sums are rounded separately (no FMA), so the
// step is reproducible from G alone.  eta_out = 1 / (2 lambda), or 0 when
// G = 0 (no step).
__global__ void lambda_max_kernel(const double* __restrict__ G, int k, double* eta_out,
                                  double* lam_out)
{
    __shared__ double x[256], y[256];
    __shared__ double lam_s;
    __shared__ int stop;
    const int tid = threadIdx.x;
    if (tid < k) x[tid] = 1.0 / sqrt((double)k);
    if (tid == 0) {
        lam_s = 0.0;
        stop = 0;
    }
    __syncthreads();
    for (int it = 0; it < 20; ++it) {
        if (tid < k) {
            double s = 0.0;
            for (int d = 0; d < k; ++d) s = __dadd_rn(s, __dmul_rn(G[tid * k + d], x[d]));
            y[tid] = s;
        }
        __syncthreads();
        if (tid == 0) {
            double nrm = 0.0;
            for (int c = 0; c < k; ++c) nrm = __dadd_rn(nrm, __dmul_rn(y[c], y[c]));
            lam_s = sqrt(nrm);
            stop = lam_s == 0.0;
        }
        __syncthreads();
        if (stop) break;
        if (tid < k) x[tid] = y[tid] / lam_s;
        __syncthreads();
    }
    if (tid == 0) {
        *lam_out = lam_s;
        *eta_out = lam_s > 0.0 ? 1.0 / (2.0 * lam_s) : 0.0;
    }
}

cudaError_t launch_lambda_max(const double* G, int k, double* eta_out, double* lam_out,
                              cudaStream_t st)
{
    if (k > 256) return cudaErrorInvalidValue;
    lambda_max_kernel<<<1, 256, 0, st>>>(G, k, eta_out, lam_out);
    return cudaGetLastError();
}

// One thread per candidate element, column-major (consecutive threads take
// consecutive rows of a column).  eta is read from device memory: either the
// caller's step or the power iteration's.
template <typename T>
__global__ void pg_apply_kernel(int64_t rows, int k, EllDev F, const double* __restrict__ Go,
                                const T* __restrict__ Y, int64_t ldy,
                                const double* __restrict__ eta_p, T* __restrict__ Xt,
                                int64_t ldx)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rows * k) return;
    const int c = (int)(g / rows);
    const int64_t r = g - (int64_t)c * rows;
    const int cnt = F.cnt[r];
    const int32_t* col = F.col + r * F.ld;
    const T* val = static_cast<const T*>(F.val) + r * F.ld;
    double s = 0.0, v = 0.0;
    for (int q = 0; q < cnt; ++q) {
        const int d = col[q];
        const double x = (double)val[q];
        if (d == c) v = x;
        s = fma(x, Go[(int64_t)d * k + c], s);
    }
    T outv = T(0);
    if (v != 0.0) {
        const double grad = 2.0 * (s - (double)Y[r * ldy + c]);
        const double x = v - *eta_p * grad;
        outv = x > 0.0 ? (T)x : T(0);
    }
    Xt[(int64_t)c * ldx + r] = outv;
}

template <typename T>
cudaError_t launch_pg_apply(int64_t rows, int k, const EllDev& F, const double* Go, const T* Y,
                            int64_t ldy, const double* eta, T* Xt, int64_t ldx, cudaStream_t st)
{
    const int64_t total = rows * k;
    if (total == 0) return cudaSuccess;
    const int B = 256;
    pg_apply_kernel<T><<<(unsigned)((total + B - 1) / B), B, 0, st>>>(rows, k, F, Go, Y, ldy, eta,
                                                                      Xt, ldx);
    return cudaGetLastError();
}

template cudaError_t launch_grad<float, float>(int64_t, int, const EllDev&, const double*, const float*, int64_t, float*, cudaStream_t);
template cudaError_t launch_grad<float, double>(int64_t, int, const EllDev&, const double*, const float*, int64_t, double*, cudaStream_t);
template cudaError_t launch_grad<double, float>(int64_t, int, const EllDev&, const double*, const double*, int64_t, float*, cudaStream_t);
template cudaError_t launch_grad<double, double>(int64_t, int, const EllDev&, const double*, const double*, int64_t, double*, cudaStream_t);
template cudaError_t launch_pg_apply<float>(int64_t, int, const EllDev&, const double*, const float*, int64_t, const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_pg_apply<double>(int64_t, int, const EllDev&, const double*, const double*, int64_t, const double*, double*, int64_t, cudaStream_t);

}  // namespace espnmf
