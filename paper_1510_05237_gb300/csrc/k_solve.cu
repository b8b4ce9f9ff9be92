// k_solve.cu -- the k x k solve and the projection of Alg. 2 steps 1 and 3:
//   X = Y (F^T F)^-1, then every entry that is not > 0 becomes +0,
// written column-major (Xt[c * ldx + row]) for the per-column selection.
//
// (F^T F)^-1 comes from the FP64 Gram inverse kernel, rounded to T, and
// stays in shared memory for all of a block's row tiles.  A tile of BM rows
// of Y is staged transposed (Ys[d][r]); each thread owns a TR-row x
// 8-column block of X (TR = 8 in FP32, 4 in FP64), so per step d it loads TR
// values of Y and 8 of the inverse (128-bit shared loads) for 8 TR FMAs.
// Columns are split over G = ceil(k/8) thread groups and rows over 256/G, so
// BM = TR * (256 / G).  A thread's rows are consecutive, so each output
// column is written with 128-bit stores.  A NaN or Inf raises ST_NONFINITE
// (and is stored as +0).
#include "common.cuh"

namespace espnmf {

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    __device__ static void load(const float* p, float v[4])
    {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
    __device__ static void store(float* p, const float v[4])
    {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<double> {
    __device__ static void load(const double* p, double v[4])
    {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static void store(double* p, const double v[4])
    {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
    }
};

// Rows of the output tile per thread: 8 in FP32 (8 x 8 accumulators), 4 in
// FP64 (its 8-byte registers would otherwise crowd out occupancy).
template <typename T> struct SolveTile { static constexpr int TR = 8; };
template <> struct SolveTile<double> { static constexpr int TR = 4; };

template <typename T>
__global__ void __launch_bounds__(256)
solve_project_kernel(const T* __restrict__ Y, int64_t ldy, int64_t rows,
                     int k, int kp8, int G, int BM,
                     const T* __restrict__ Ginv, T* __restrict__ Xt,
                     int64_t ldx, unsigned* status)
{
    constexpr int TR = SolveTile<T>::TR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Gs = reinterpret_cast<T*>(smem_raw);   // [k][kp8]
    T* Ys = Gs + (size_t)k * kp8;             // [k][BM]
    const int tid = threadIdx.x;
    for (int e = tid; e < k * kp8; e += blockDim.x) {
        const int d = e / kp8, c = e - d * kp8;
        Gs[e] = c < k ? Ginv[d * k + c] : T(0);
    }
    const int g = tid % G;
    const int rg = tid / G;
    const bool active = rg < BM / TR;
    bool bad = false;
    for (int64_t r0 = (int64_t)blockIdx.x * BM; r0 < rows; r0 += (int64_t)gridDim.x * BM) {
        __syncthreads();
        const int nr = (int)(rows - r0 < BM ? rows - r0 : BM);
        // thread rr stages row rr: consecutive threads write consecutive
        // addresses of each Ys[d][.] line (no bank conflicts)
        for (int rr = tid; rr < BM; rr += blockDim.x) {
            const T* yr = Y + (r0 + rr) * ldy;
            for (int d0 = 0; d0 < k; d0 += 4) {
                T v[4];
                if (rr < nr) Vec4<T>::load(yr + d0, v);
                else v[0] = v[1] = v[2] = v[3] = T(0);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (d0 + u < k) Ys[(d0 + u) * BM + rr] = v[u];
            }
        }
        __syncthreads();
        if (active) {
            T acc[TR][8];
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[r][j] = T(0);
            for (int d = 0; d < k; ++d) {
                T y[TR], ga[4], gb[4];
#pragma unroll
                for (int h = 0; h < TR; h += 4) Vec4<T>::load(Ys + d * BM + rg * TR + h, y + h);
                Vec4<T>::load(Gs + d * kp8 + g * 8, ga);
                Vec4<T>::load(Gs + d * kp8 + g * 8 + 4, gb);
#pragma unroll
                for (int r = 0; r < TR; ++r) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[r][j] += y[r] * ga[j];
                        acc[r][4 + j] += y[r] * gb[j];
                    }
                }
            }
            const int row0 = rg * TR;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = g * 8 + j;
                if (c >= k) continue;
                T x[TR];
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const T v = acc[r][j];
                    if (!isfinite(v)) bad = true;
                    x[r] = v > T(0) ? v : T(0);
                }
                T* dst = Xt + (int64_t)c * ldx + r0 + row0;
                if (row0 + TR <= nr) {
#pragma unroll
                    for (int h = 0; h < TR; h += 4) Vec4<T>::store(dst + h, x + h);
                } else {
                    for (int r = 0; r < TR; ++r)
                        if (row0 + r < nr) dst[r] = x[r];
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

template <typename T>
cudaError_t launch_solve(const T* Y, int64_t ldy, int64_t rows, int k,
                         const T* Ginv, T* Xt, int64_t ldx, unsigned* status,
                         cudaStream_t st, int sm_count)
{
    constexpr int TR = SolveTile<T>::TR;
    if (rows == 0) return cudaSuccess;
    const int kp8 = (k + 7) / 8 * 8;
    const int G = kp8 / 8;
    int R = 256 / G;                          // row groups of TR rows
    // keep the staged tile within budget
    while (R > 1 && ((size_t)k * kp8 + (size_t)k * TR * R) * sizeof(T) > 200 * 1024) R /= 2;
    const int BM = TR * R;
    const size_t smem = ((size_t)k * kp8 + (size_t)k * BM) * sizeof(T);
    int64_t tiles = (rows + BM - 1) / BM;
    int64_t grid = (int64_t)sm_count * 2;
    if (grid > tiles) grid = tiles;
    solve_project_kernel<T><<<(unsigned)grid, 256, smem, st>>>(
        Y, ldy, rows, k, kp8, G, BM, Ginv, Xt, ldx, status);
    return cudaGetLastError();
}

cudaError_t setup_solve()
{
    cudaError_t e = cudaFuncSetAttribute(solve_project_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(solve_project_kernel<double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
}

template cudaError_t launch_solve<float>(const float*, int64_t, int64_t, int, const float*, float*, int64_t, unsigned*, cudaStream_t, int);
template cudaError_t launch_solve<double>(const double*, int64_t, int64_t, int, const double*, double*, int64_t, unsigned*, cudaStream_t, int);

}  // namespace espnmf
