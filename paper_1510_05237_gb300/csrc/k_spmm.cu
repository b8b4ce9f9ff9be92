// k_spmm.cu -- the sparse products of Alg. 2 steps 1 and 3:
//   Y = A^T U (V half)   and   Y = A V (U half).
//
// A is streamed once per product from a sliced-ELLPACK layout (SELL-32):
// a warp's 32 lanes walk 32 segments of about the same length, so every
// load of A is a coalesced 128-byte transaction.  A row is cut into 1..32
// segments of at most 64 entries held by adjacent lanes; each lane sums its
// segment and the lanes of a row are combined by a fixed shuffle tree.
//
// The factor F is gathered two ways, chosen per factor row:
//   heavy rows (cnt >= heavy, nearly dense): the dense copy of the row is
//     read with 128-bit loads into KP register accumulators;
//   light rows: the row's (column, value) pairs, read as 128-bit vectors,
//     are added into per-thread accumulators in shared memory, slot c of
//     thread tid at acc[c * blockDim + tid] -- a warp's lanes always touch
//     32 distinct banks whatever columns they update.
// Enforced-sparse factors of text data are both: most rows hold a few
// nonzeros, while the rows of the most frequent terms end up in almost every
// column's top-t.  The loop is software-pipelined: while a step's gathers
// run, the next step's factor-row counts and the step after's entries of A
// are already in flight.  Sums are taken in a fixed order (storage order per
// lane, a fixed tree across lanes, chunk order for very long rows), so the
// product is bitwise reproducible.
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
    const int32_t* seg_grp;
    const int32_t* fcnt;
    const int32_t* fcol;
    const T* fval;
    const T* fdense;
    int heavy;
    int k;
    T* Y;        // rows x KP (ldy == KP)
    T* partials; // npart x KP
};

// FP32: heavy rows into KP registers, light pairs into shared memory.
template <int KP>
__global__ void __launch_bounds__(256)
spmm_sell_f32_kernel(SpmmParams<float> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* slots = reinterpret_cast<float*>(smem_raw);
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int64_t s = (int64_t)blockIdx.x * (B >> 5) + (tid >> 5);
    if (s >= p.nslices) return;
    const int64_t seg = s * 32 + lane;
    float acc[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) acc[c] = 0.f;
    float* my = slots + tid;
#pragma unroll 4
    for (int c = 0; c < KP; ++c) my[c * B] = 0.f;

    const int len = p.slice_len[s];
    const int64_t base = p.slice_ptr[s] + lane;
    const int32_t* __restrict__ idx = p.idx + base;
    const float* __restrict__ val = p.val + base;
    const int32_t* __restrict__ fcnt = p.fcnt;
    const int heavy = p.heavy;

    auto gather = [&](int i, float a, int cnt) {
        if (cnt >= heavy) {
            const float4* r = reinterpret_cast<const float4*>(p.fdense + (int64_t)i * KP);
#pragma unroll
            for (int q = 0; q < KP / 4; ++q) {
                const float4 v = __ldg(r + q);
                acc[4 * q + 0] = fmaf(a, v.x, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(a, v.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(a, v.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(a, v.w, acc[4 * q + 3]);
            }
        } else if (cnt > 0) {
            const int4* cr = reinterpret_cast<const int4*>(p.fcol + (int64_t)i * KP);
            const float4* vr = reinterpret_cast<const float4*>(p.fval + (int64_t)i * KP);
            for (int q = 0; q < cnt; q += 4) {
                const int4 cc = __ldg(cr + (q >> 2));
                const float4 vv = __ldg(vr + (q >> 2));
                my[cc.x * B] = fmaf(a, vv.x, my[cc.x * B]);
                if (q + 1 < cnt) my[cc.y * B] = fmaf(a, vv.y, my[cc.y * B]);
                if (q + 2 < cnt) my[cc.z * B] = fmaf(a, vv.z, my[cc.z * B]);
                if (q + 3 < cnt) my[cc.w * B] = fmaf(a, vv.w, my[cc.w * B]);
            }
        }
    };
    auto load2 = [&](int pp, int& i0, float& a0, int& i1, float& a1) {
        i0 = pp < len ? __ldcs(idx + (int64_t)pp * 32) : -1;
        a0 = pp < len ? __ldcs(val + (int64_t)pp * 32) : 0.f;
        i1 = pp + 1 < len ? __ldcs(idx + (int64_t)(pp + 1) * 32) : -1;
        a1 = pp + 1 < len ? __ldcs(val + (int64_t)(pp + 1) * 32) : 0.f;
    };

    // stage j: entries (j, j+1) gathered; stage j+2's counts and j+4's
    // entries are loaded meanwhile
    int i0, i1, n0, n1;
    float a0, a1, b0, b1;
    load2(0, i0, a0, i1, a1);
    load2(2, n0, b0, n1, b1);
    int c0 = i0 >= 0 ? __ldg(fcnt + i0) : 0;
    int c1 = i1 >= 0 ? __ldg(fcnt + i1) : 0;
    for (int p0 = 0; p0 < len; p0 += 2) {
        const int d0 = n0 >= 0 ? __ldg(fcnt + n0) : 0;
        const int d1 = n1 >= 0 ? __ldg(fcnt + n1) : 0;
        int m0, m1;
        float e0, e1;
        load2(p0 + 4, m0, e0, m1, e1);
        gather(i0, a0, c0);
        gather(i1, a1, c1);
        i0 = n0; i1 = n1; a0 = b0; a1 = b1; c0 = d0; c1 = d1;
        n0 = m0; n1 = m1; b0 = e0; b1 = e1;
    }

#pragma unroll
    for (int c = 0; c < KP; ++c) acc[c] += my[c * B];
    // combine the lanes [head, end) of each row: fixed tree, lane head
    // ends with the row's sum
    const int grp = p.seg_grp[seg];
    const int head = grp >> 8, end = grp & 0xff;
    const int maxg = __reduce_max_sync(0xffffffffu, (unsigned)(end - head));
    for (int off = 1; off < maxg; off <<= 1) {
        const bool take = lane + off < end;
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            const float v = __shfl_down_sync(0xffffffffu, acc[c], off);
            if (take) acc[c] += v;
        }
    }
    const int row = p.seg_row[seg];
    if (row < 0 || lane != head) return;
    const int part = p.seg_part[seg];
    float* out = part < 0 ? p.Y + (int64_t)row * KP : p.partials + (int64_t)part * KP;
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int q = 0; q < KP / 4; ++q)
        o4[q] = make_float4(acc[4 * q + 0], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

// FP64 (the plain form): every gather into shared-memory accumulators.
__global__ void __launch_bounds__(256)
spmm_sell_f64_kernel(SpmmParams<double> p, int KP)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* slots = reinterpret_cast<double*>(smem_raw);
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int64_t s = (int64_t)blockIdx.x * (B >> 5) + (tid >> 5);
    if (s >= p.nslices) return;
    const int64_t seg = s * 32 + lane;
    double* my = slots + tid;
    for (int c = 0; c < KP; ++c) my[c * B] = 0.0;
    const int len = p.slice_len[s];
    const int64_t base = p.slice_ptr[s] + lane;
    const int heavy = p.heavy;
    for (int p0 = 0; p0 < len; ++p0) {
        const int i = __ldcs(p.idx + base + (int64_t)p0 * 32);
        const double a = __ldcs(p.val + base + (int64_t)p0 * 32);
        const int cnt = i >= 0 ? __ldg(p.fcnt + i) : 0;
        if (cnt >= heavy) {
            const double2* r = reinterpret_cast<const double2*>(p.fdense + (int64_t)i * KP);
            for (int q = 0; q < (p.k + 1) / 2; ++q) {
                const double2 v = __ldg(r + q);
                my[(2 * q) * B] = fma(a, v.x, my[(2 * q) * B]);
                my[(2 * q + 1) * B] = fma(a, v.y, my[(2 * q + 1) * B]);
            }
        } else if (cnt > 0) {
            const int4* cr = reinterpret_cast<const int4*>(p.fcol + (int64_t)i * KP);
            const double2* vr = reinterpret_cast<const double2*>(p.fval + (int64_t)i * KP);
            for (int q = 0; q < cnt; q += 4) {
                const int4 cc = __ldg(cr + (q >> 2));
                const double2 v01 = __ldg(vr + (q >> 1));
                const double2 v23 = __ldg(vr + (q >> 1) + 1);
                my[cc.x * B] = fma(a, v01.x, my[cc.x * B]);
                if (q + 1 < cnt) my[cc.y * B] = fma(a, v01.y, my[cc.y * B]);
                if (q + 2 < cnt) my[cc.z * B] = fma(a, v23.x, my[cc.z * B]);
                if (q + 3 < cnt) my[cc.w * B] = fma(a, v23.y, my[cc.w * B]);
            }
        }
    }
    const int grp = p.seg_grp[seg];
    const int head = grp >> 8, end = grp & 0xff;
    const int maxg = __reduce_max_sync(0xffffffffu, (unsigned)(end - head));
    const int row = p.seg_row[seg];
    const int part = p.seg_part[seg];
    double* out = (row >= 0 && lane == head)
                      ? (part < 0 ? p.Y + (int64_t)row * KP : p.partials + (int64_t)part * KP)
                      : nullptr;
    for (int c = 0; c < KP; ++c) {
        double v = my[c * B];
        for (int off = 1; off < maxg; off <<= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, off);
            if (lane + off < end) v += w;
        }
        if (out) out[c] = v;
    }
}

// One warp per split row: Y[row] = sum of its segments' partials, in order.
template <typename T>
__global__ void spmm_combine_kernel(int64_t nsplit, const int32_t* split_row,
                                    const int32_t* split_first,
                                    const int32_t* split_count,
                                    const T* partials, int KP, T* Y)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nsplit) return;
    const int row = split_row[w];
    const int first = split_first[w];
    const int count = split_count[w];
    for (int c = lane; c < KP; c += 32) {
        T s0 = T(0);
        const T* pp = partials + (int64_t)first * KP + c;
        for (int q = 0; q < count; ++q) s0 += pp[(int64_t)q * KP];
        Y[(int64_t)row * KP + c] = s0;
    }
}

static int spmm_block(int KP, size_t esz, size_t limit)
{
    // KP shared slots per thread, at most `limit` bytes per block.
    int b = (int)(limit / ((size_t)KP * esz));
    b = (b / 32) * 32;
    if (b > 256) b = 256;
    if (b < 32) b = 32;
    return b;
}

template <int KP>
static cudaError_t launch_f32(const SpmmParams<float>& p, int64_t nslices, cudaStream_t st)
{
    const int B = spmm_block(KP, 4, 48 * 1024);
    const size_t smem = (size_t)KP * B * 4;
    const int64_t wpb = B / 32;
    const int64_t grid = (nslices + wpb - 1) / wpb;
    spmm_sell_f32_kernel<KP><<<(unsigned)grid, B, smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmm(const SellDev& S, const EllDev& F, int k, T* Y,
                        int64_t ldy, cudaStream_t st, int sm_count)
{
    (void)sm_count;
    (void)ldy;
    if (S.nslices == 0) return cudaSuccess;
    SpmmParams<T> p;
    p.nslices = S.nslices;
    p.slice_ptr = S.slice_ptr;
    p.slice_len = S.slice_len;
    p.idx = S.idx;
    p.val = static_cast<const T*>(S.val);
    p.seg_row = S.seg_row;
    p.seg_part = S.seg_part;
    p.seg_grp = S.seg_grp;
    p.fcnt = F.cnt;
    p.fcol = F.col;
    p.fval = static_cast<const T*>(F.val);
    p.fdense = static_cast<const T*>(F.dense);
    p.heavy = F.heavy;
    p.k = k;
    p.Y = Y;
    p.partials = static_cast<T*>(S.partials);
    const int KP = F.ld;
    if constexpr (sizeof(T) == 4) {
        switch (KP) {
#define ESPNMF_KP(v) case v: return launch_f32<v>(p, S.nslices, st);
            ESPNMF_KP(4) ESPNMF_KP(8) ESPNMF_KP(12) ESPNMF_KP(16) ESPNMF_KP(20) ESPNMF_KP(24)
            ESPNMF_KP(28) ESPNMF_KP(32) ESPNMF_KP(36) ESPNMF_KP(40) ESPNMF_KP(44) ESPNMF_KP(48)
            ESPNMF_KP(52) ESPNMF_KP(56) ESPNMF_KP(60) ESPNMF_KP(64) ESPNMF_KP(80) ESPNMF_KP(96)
            ESPNMF_KP(112) ESPNMF_KP(128)
#undef ESPNMF_KP
        default: return cudaErrorInvalidValue;
        }
    } else {
        const int B = spmm_block(KP, 8, 96 * 1024);
        const size_t smem = (size_t)KP * B * 8;
        const int64_t wpb = B / 32;
        const int64_t grid = (S.nslices + wpb - 1) / wpb;
        spmm_sell_f64_kernel<<<(unsigned)grid, B, smem, st>>>(p, KP);
        return cudaGetLastError();
    }
}

template <typename T>
cudaError_t launch_spmm_combine(const SellDev& S, int KP, T* Y, int64_t ldy,
                                cudaStream_t st)
{
    (void)ldy;
    if (S.nsplit == 0) return cudaSuccess;
    const int B = 256;
    const int64_t grid = (S.nsplit * 32 + B - 1) / B;
    spmm_combine_kernel<T><<<(unsigned)grid, B, 0, st>>>(
        S.nsplit, S.split_row, S.split_first, S.split_count,
        static_cast<const T*>(S.partials), KP, Y);
    return cudaGetLastError();
}

cudaError_t setup_spmm()
{
    return cudaFuncSetAttribute(spmm_sell_f64_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
}

template cudaError_t launch_spmm<float>(const SellDev&, const EllDev&, int, float*, int64_t, cudaStream_t, int);
template cudaError_t launch_spmm<double>(const SellDev&, const EllDev&, int, double*, int64_t, cudaStream_t, int);
template cudaError_t launch_spmm_combine<float>(const SellDev&, int, float*, int64_t, cudaStream_t);
template cudaError_t launch_spmm_combine<double>(const SellDev&, int, double*, int64_t, cudaStream_t);

}  // namespace espnmf
