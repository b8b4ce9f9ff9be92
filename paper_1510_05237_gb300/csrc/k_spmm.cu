// k_spmm.cu -- the sparse products of Alg. 2 steps 1 and 3:
//   Y = A^T U (V half)   and   Y = A V (U half).
//
// A is streamed once per product from a sliced-ELLPACK layout (SELL-32,
// segments sorted by length, so a warp's 32 lanes walk 32 segments of equal
// length and every load of A is a coalesced 128-byte transaction).  The
// factor is gathered from its row-packed sparse form: for a stored a_ij the
// thread reads row j of the factor -- only its nonzeros, cnt[j] pairs -- and
// adds a_ij * f_jc into its private accumulator for column c.
//
// Accumulators live in shared memory, k slots per thread, slot c of thread
// tid at acc[c * blockDim + tid]: lanes of a warp always touch 32 distinct
// banks whatever columns they update.  Each thread sums its segment in the
// stored order and segments of a split row are added in segment order by
// spmm_combine, so the product is bitwise reproducible.
#include "common.cuh"

namespace espnmf {

template <typename T>
struct SpmmParams {
    int64_t nslices;
    const int64_t* slice_ptr;
    const int32_t* slice_len;
    const int32_t* idx;
    const T* val;
    const int32_t* seg_row;
    const int32_t* seg_part;
    const int32_t* fcnt;
    const int32_t* fcol;
    const T* fval;
    int k;
    T* Y;
    int64_t ldy;
    T* partials;
};

template <typename T>
__global__ void __launch_bounds__(256)
spmm_sell_kernel(SpmmParams<T> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int64_t s = (int64_t)blockIdx.x * (B >> 5) + (tid >> 5);
    if (s >= p.nslices) return;
    const int64_t seg = s * 32 + lane;
    const int row = p.seg_row[seg];
    const int k = p.k;
    T* my = acc + tid;
    for (int c = 0; c < k; ++c) my[c * B] = T(0);

    const int len = p.slice_len[s];
    const int64_t base = p.slice_ptr[s] + lane;
    const int32_t* __restrict__ idx = p.idx + base;
    const T* __restrict__ val = p.val + base;
    const int32_t* __restrict__ fcnt = p.fcnt;
    const int32_t* __restrict__ fcol = p.fcol;
    const T* __restrict__ fval = p.fval;

    // Four stored entries per step: their factor-row lookups are issued
    // together so the dependent gathers overlap.
    for (int p0 = 0; p0 < len; p0 += 4) {
        int i[4];
        T a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int pp = p0 + u;
            i[u] = pp < len ? __ldcs(idx + (int64_t)pp * 32) : -1;
            a[u] = pp < len ? __ldcs(val + (int64_t)pp * 32) : T(0);
        }
        int cnt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cnt[u] = i[u] >= 0 ? __ldg(fcnt + i[u]) : 0;
        int c0[4];
        T v0[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t fb = (int64_t)(i[u] >= 0 ? i[u] : 0) * k;
            c0[u] = cnt[u] > 0 ? __ldg(fcol + fb) : 0;
            v0[u] = cnt[u] > 0 ? __ldg(fval + fb) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (cnt[u] <= 0) continue;
            my[c0[u] * B] += a[u] * v0[u];
            const int64_t fb = (int64_t)i[u] * k;
            for (int q = 1; q < cnt[u]; ++q) {
                const int c = __ldg(fcol + fb + q);
                my[c * B] += a[u] * __ldg(fval + fb + q);
            }
        }
    }

    if (row < 0) return;
    const int part = p.seg_part[seg];
    T* out = part < 0 ? p.Y + (int64_t)row * p.ldy : p.partials + (int64_t)part * k;
    for (int c = 0; c < k; ++c) out[c] = my[c * B];
}

// One warp per split row: Y[row] = sum of its segments' partials, in order.
template <typename T>
__global__ void spmm_combine_kernel(int64_t nsplit, const int32_t* split_row,
                                    const int32_t* split_first,
                                    const int32_t* split_count,
                                    const T* partials, int k, T* Y,
                                    int64_t ldy)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nsplit) return;
    const int row = split_row[w];
    const int first = split_first[w];
    const int count = split_count[w];
    for (int c = lane; c < k; c += 32) {
        T s = T(0);
        const T* pp = partials + (int64_t)first * k + c;
        for (int q = 0; q < count; ++q) s += pp[(int64_t)q * k];
        Y[(int64_t)row * ldy + c] = s;
    }
}

static int spmm_block(int k, size_t esz)
{
    // k slots per thread; keep a block within 96 KB so two fit on an SM.
    int b = (int)((96 * 1024) / ((size_t)k * esz));
    b = (b / 32) * 32;
    if (b > 256) b = 256;
    if (b < 32) b = 32;
    return b;
}

template <typename T>
cudaError_t launch_spmm(const SellDev& S, const EllDev& F, int k, T* Y,
                        int64_t ldy, cudaStream_t st, int sm_count)
{
    (void)sm_count;
    if (S.nslices == 0) return cudaSuccess;
    SpmmParams<T> p;
    p.nslices = S.nslices;
    p.slice_ptr = S.slice_ptr;
    p.slice_len = S.slice_len;
    p.idx = S.idx;
    p.val = static_cast<const T*>(S.val);
    p.seg_row = S.seg_row;
    p.seg_part = S.seg_part;
    p.fcnt = F.cnt;
    p.fcol = F.col;
    p.fval = static_cast<const T*>(F.val);
    p.k = k;
    p.Y = Y;
    p.ldy = ldy;
    p.partials = static_cast<T*>(S.partials);
    const int B = spmm_block(k, sizeof(T));
    const size_t smem = (size_t)k * B * sizeof(T);
    const int64_t wpb = B / 32;
    const int64_t grid = (S.nslices + wpb - 1) / wpb;
    spmm_sell_kernel<T><<<(unsigned)grid, B, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmm_combine(const SellDev& S, int k, T* Y, int64_t ldy,
                                cudaStream_t st)
{
    if (S.nsplit == 0) return cudaSuccess;
    const int B = 256;
    const int64_t grid = (S.nsplit * 32 + B - 1) / B;
    spmm_combine_kernel<T><<<(unsigned)grid, B, 0, st>>>(
        S.nsplit, S.split_row, S.split_first, S.split_count,
        static_cast<const T*>(S.partials), k, Y, ldy);
    return cudaGetLastError();
}

cudaError_t setup_spmm()
{
    cudaError_t e = cudaFuncSetAttribute(spmm_sell_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(spmm_sell_kernel<double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template cudaError_t launch_spmm<float>(const SellDev&, const EllDev&, int, float*, int64_t, cudaStream_t, int);
template cudaError_t launch_spmm<double>(const SellDev&, const EllDev&, int, double*, int64_t, cudaStream_t, int);
template cudaError_t launch_spmm_combine<float>(const SellDev&, int, float*, int64_t, cudaStream_t);
template cudaError_t launch_spmm_combine<double>(const SellDev&, int, double*, int64_t, cudaStream_t);

}  // namespace espnmf
