// k_solve.cu -- the k x k solve and the projection of Alg. 2 steps 1 and 3:
//   X = Y (F^T F)^-1, then every entry that is not > 0 becomes +0,
// written column-major (Xt[c * ldx + row]) for the per-column selection.
//
// (F^T F)^-1 comes from the FP64 Cholesky kernel, rounded to T.  A block
// keeps it in shared memory for all its row tiles; each tile of BM rows of Y
// is staged transposed (Ys[d][r]) so that thread r reads its own row without
// bank conflicts while the 8 inverse entries it multiplies by are broadcast.
// A NaN or Inf raises ST_NONFINITE (and is stored as +0).
#include "common.cuh"

namespace espnmf {

template <typename T, int BM>
__global__ void __launch_bounds__(256)
solve_project_kernel(const T* __restrict__ Y, int64_t ldy, int64_t rows,
                     int k, int kp, const T* __restrict__ Ginv,
                     T* __restrict__ Xt, int64_t ldx, unsigned* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Gs = reinterpret_cast<T*>(smem_raw);   // [k][kp]
    T* Ys = Gs + (size_t)k * kp;              // [k][BM+1]
    const int tid = threadIdx.x;
    for (int e = tid; e < k * kp; e += blockDim.x) {
        const int d = e / kp, c = e - d * kp;
        Gs[e] = c < k ? Ginv[d * k + c] : T(0);
    }
    const int r = tid % BM;
    const int g = tid / BM;
    const int G = blockDim.x / BM;
    bool bad = false;
    for (int64_t r0 = (int64_t)blockIdx.x * BM; r0 < rows; r0 += (int64_t)gridDim.x * BM) {
        __syncthreads();
        const int nr = (int)(rows - r0 < BM ? rows - r0 : BM);
        for (int e = tid; e < BM * k; e += blockDim.x) {
            const int rr = e / k, d = e - rr * k;
            Ys[d * (BM + 1) + rr] = rr < nr ? Y[(r0 + rr) * ldy + d] : T(0);
        }
        __syncthreads();
        for (int cb = g * 8; cb < k; cb += G * 8) {
            T acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = T(0);
            for (int d = 0; d < k; ++d) {
                const T y = Ys[d * (BM + 1) + r];
                const T* gr = Gs + d * kp + cb;
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] += y * gr[j];
            }
            if (r < nr) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = cb + j;
                    if (c < k) {
                        T x = acc[j];
                        if (!isfinite(x)) bad = true;
                        Xt[(int64_t)c * ldx + r0 + r] = x > T(0) ? x : T(0);
                    }
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

template <typename T>
static constexpr int solve_bm() { return sizeof(T) == 8 ? 64 : 128; }

template <typename T>
cudaError_t launch_solve(const T* Y, int64_t ldy, int64_t rows, int k,
                         const T* Ginv, T* Xt, int64_t ldx, unsigned* status,
                         cudaStream_t st, int sm_count)
{
    if (rows == 0) return cudaSuccess;
    constexpr int BM = solve_bm<T>();
    const int kp = (k + 7) / 8 * 8;
    const size_t smem = ((size_t)k * kp + (size_t)k * (BM + 1)) * sizeof(T);
    int64_t tiles = (rows + BM - 1) / BM;
    int64_t grid = (int64_t)sm_count * 2;
    if (grid > tiles) grid = tiles;
    solve_project_kernel<T, BM><<<(unsigned)grid, 256, smem, st>>>(
        Y, ldy, rows, k, kp, Ginv, Xt, ldx, status);
    return cudaGetLastError();
}

cudaError_t setup_solve()
{
    cudaError_t e = cudaFuncSetAttribute(solve_project_kernel<float, 128>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(solve_project_kernel<double, 64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

template cudaError_t launch_solve<float>(const float*, int64_t, int64_t, int, const float*, float*, int64_t, unsigned*, cudaStream_t, int);
template cudaError_t launch_solve<double>(const double*, int64_t, int64_t, int, const double*, double*, int64_t, unsigned*, cudaStream_t, int);

}  // namespace espnmf
