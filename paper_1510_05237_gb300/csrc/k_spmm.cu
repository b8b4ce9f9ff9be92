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
//   light rows (fewer than `heavy` nonzeros, most rows of an enforced-sparse
//     factor): one 16-byte record holds the row's count and its first three
//     (column, value) pairs, so a row of up to three nonzeros costs a single
//     load; each value is added into a per-thread accumulator in shared
//     memory, slot c of thread tid at acc[c * blockDim + tid] -- a warp's
//     lanes always touch 32 distinct banks whatever columns they update;
//   heavy rows (nearly dense: the rows of the most frequent terms end up in
//     almost every column's top-t): each lane reads its own entry's row
//     from the row's dense copy (16-byte loads) into register accumulators.
// The number of warps that share a slice's columns (1, 2 or 4: fewer
// registers and slots per thread, so more warps in flight) and the launch's
// shared-memory carveout (the rest of the SM's memory is L1, which holds the
// heavy rows) are a launch shape (SpmmConfig) timed by the host; all shapes
// add the same products in the same order, so the result does not depend
// on the choice.
// The loop is software-pipelined: while a step's gathers run, the records
// of the next step and the entries of A of the next two are in flight, and
// the slice's whole run of A is prefetched into the L2 when the warp starts
// (deeper register pipelines measured slower: they cost registers the heavy
// gathers need).
// Sums are taken in a fixed order (storage order per lane, a fixed tree
// across lanes, chunk order for very long rows), so the product is bitwise
// reproducible.
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
    const uint4* frec;
    int dld;
    int fld;
    int heavy;
    int k;
    T* Y;        // rows x KP (ldy == KP)
    T* partials; // npart x KP
};

// FP32.  NS warps share a slice: warp h of the NS owns the output columns
// [h * CW, min(KP, (h + 1) * CW)), CW = KP / NS rounded up to 4, for all 32
// segments of the slice.  Each warp streams the slice's entries of A (the
// NS warps read the same lines, mostly from L1), adds its columns of light
// rows' values into its shared-memory slots and gathers its CW columns of
// heavy rows (CW / 4 16-byte loads) into CW register accumulators.  A larger
// NS means fewer registers and slots per thread, so more warps in flight
// for the same shared memory, at the price of re-reading A and the records.
// Every NS adds the same products in the same order.
template <int KP, int NS>
struct SplitShape {
    static constexpr int CW = ((KP + NS - 1) / NS + 3) / 4 * 4;
};

template <int KP, int NS>
__global__ void __launch_bounds__(256, KP > 64 ? 1 : 2)
spmm_sell_f32_kernel(SpmmParams<float> p)
{
    constexpr int CW = SplitShape<KP, NS>::CW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int h = warp % NS;                  // column block of this warp
    const int c0 = h * CW;
    const int cw = KP - c0 < CW ? KP - c0 : CW;   // columns owned (> 0, multiple of 4)
    float* slots = reinterpret_cast<float*>(smem_raw);                   // CW x B
    const int64_t s = (int64_t)blockIdx.x * (B >> 5) / NS + warp / NS;
    if (s >= p.nslices || cw <= 0) return;
    const int64_t seg = s * 32 + lane;

    float acc[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = 0.f;
    float* my = slots + tid;
#pragma unroll 4
    for (int c = 0; c < CW; ++c) my[c * B] = 0.f;

    const int len = p.slice_len[s];
    const int64_t base = p.slice_ptr[s] + lane;
    const int32_t* __restrict__ idx = p.idx + base;
    const float* __restrict__ val = p.val + base;
    const uint4* __restrict__ rec = p.frec;
    const float4* __restrict__ dense4 = reinterpret_cast<const float4*>(p.fdense) + c0 / 4;
    const int dld4 = p.dld / 4;
    const int heavy = p.heavy;
    const int fld = p.fld;
    const unsigned ucw = (unsigned)cw;

    // one value of a light row: column c (absolute) if this warp owns it
    auto add = [&](unsigned c, float x) {
        const unsigned r = c - (unsigned)c0;
        if (r < ucw) my[r * B] += x;
    };
    auto light = [&](int i, float a, const uint4& r) {
        const int cnt = record_cnt(r.x);
        if (cnt == 0 || cnt >= heavy) return;
        add((r.x >> 8) & 0xffu, a * __uint_as_float(r.y));
        if (cnt > 1) add((r.x >> 16) & 0xffu, a * __uint_as_float(r.z));
        if (cnt > 2) add(r.x >> 24, a * __uint_as_float(r.w));
        if (cnt > 3) {
            const int32_t* cr = p.fcol + (int64_t)i * fld;
            const float* vr = p.fval + (int64_t)i * fld;
            add((unsigned)__ldg(cr + 3), a * __ldg(vr + 3));
            for (int q = 4; q < cnt; q += 4) {
                const int4 cc = __ldg(reinterpret_cast<const int4*>(cr + q));
                const float4 vv = __ldg(reinterpret_cast<const float4*>(vr + q));
                add((unsigned)cc.x, a * vv.x);
                if (q + 1 < cnt) add((unsigned)cc.y, a * vv.y);
                if (q + 2 < cnt) add((unsigned)cc.z, a * vv.z);
                if (q + 3 < cnt) add((unsigned)cc.w, a * vv.w);
            }
        }
    };
    // this lane's heavy entry: its CW columns of the dense row
    auto heavy_row = [&](int i, float a) {
        const float4* r = dense4 + (int64_t)i * dld4;
#pragma unroll
        for (int q = 0; q < CW / 4; ++q) {
            if (4 * q >= cw) break;
            const float4 v = __ldg(r + q);
            acc[4 * q + 0] = fmaf(a, v.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(a, v.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(a, v.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(a, v.w, acc[4 * q + 3]);
        }
    };
    auto load2 = [&](int pp, int* ii, float* aa) {
        ii[0] = pp < len ? __ldcs(idx + (int64_t)pp * 32) : -1;
        aa[0] = pp < len ? __ldcs(val + (int64_t)pp * 32) : 0.f;
        ii[1] = pp + 1 < len ? __ldcs(idx + (int64_t)(pp + 1) * 32) : -1;
        aa[1] = pp + 1 < len ? __ldcs(val + (int64_t)(pp + 1) * 32) : 0.f;
    };
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    auto rec2 = [&](const int* ii, uint4* rr) {
        rr[0] = ii[0] >= 0 ? __ldg(rec + ii[0]) : zero4;
        rr[1] = ii[1] >= 0 ? __ldg(rec + ii[1]) : zero4;
    };

    // The slice's entries of A are one contiguous run per array: ask the
    // L2 for all of it now, so that the loads below wait on the L2 rather
    // than on HBM.
    if (lane == 0 && len > 0) {
        const unsigned bytes = (unsigned)len * 128u;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                     :: "l"(p.idx + p.slice_ptr[s]), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                     :: "l"(p.val + p.slice_ptr[s]), "r"(bytes) : "memory");
    }

    // Step pairs in flight: entries of A for the next DA pairs, records
    // (which need the entries' row index) for the next DR pairs.
    constexpr int DA = 2, DR = 1;
    int I[DA][2];
    float Av[DA][2];
    uint4 Rc[DR][2];
#pragma unroll
    for (int q = 0; q < DA; ++q) load2(2 * q, I[q], Av[q]);
#pragma unroll
    for (int q = 0; q < DR; ++q) rec2(I[q], Rc[q]);
    for (int p0 = 0; p0 < len; p0 += 2) {
        int ni[2];
        float na[2];
        uint4 nr[2];
        load2(p0 + 2 * DA, ni, na);
        rec2(I[DR], nr);
        light(I[0][0], Av[0][0], Rc[0][0]);
        light(I[0][1], Av[0][1], Rc[0][1]);
        if (record_cnt(Rc[0][0].x) >= heavy) heavy_row(I[0][0], Av[0][0]);
        if (record_cnt(Rc[0][1].x) >= heavy) heavy_row(I[0][1], Av[0][1]);
#pragma unroll
        for (int q = 0; q < DA - 1; ++q) {
            I[q][0] = I[q + 1][0];
            I[q][1] = I[q + 1][1];
            Av[q][0] = Av[q + 1][0];
            Av[q][1] = Av[q + 1][1];
        }
        I[DA - 1][0] = ni[0];
        I[DA - 1][1] = ni[1];
        Av[DA - 1][0] = na[0];
        Av[DA - 1][1] = na[1];
#pragma unroll
        for (int q = 0; q < DR - 1; ++q) {
            Rc[q][0] = Rc[q + 1][0];
            Rc[q][1] = Rc[q + 1][1];
        }
        Rc[DR - 1][0] = nr[0];
        Rc[DR - 1][1] = nr[1];
    }

#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] += c < cw ? my[c * B] : 0.f;
    // combine the lanes [head, end) of each row: fixed tree, lane head
    // ends with the row's sum
    const int grp = p.seg_grp[seg];
    const int head = grp >> 8, end = grp & 0xff;
    const int maxg = __reduce_max_sync(FULL, (unsigned)(end - head));
    for (int off = 1; off < maxg; off <<= 1) {
        const bool take = lane + off < end;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const float v = __shfl_down_sync(FULL, acc[c], off);
            if (take) acc[c] += v;
        }
    }
    const int row = p.seg_row[seg];
    if (row < 0 || lane != head) return;
    const int part = p.seg_part[seg];
    float* out = (part < 0 ? p.Y + (int64_t)row * KP : p.partials + (int64_t)part * KP) + c0;
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int q = 0; q < CW / 4; ++q)
        if (4 * q < cw)
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
            const double2* r = reinterpret_cast<const double2*>(p.fdense + (int64_t)i * p.dld);
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

template <int KP, int NS>
static cudaError_t launch_f32_split(const SpmmParams<float>& p, int64_t nslices, int carveout,
                                    cudaStream_t st)
{
    constexpr int CW = SplitShape<KP, NS>::CW;
    // NS warps per slice; about 48 KB of slots per block
    int B = spmm_block(CW, 4, 48 * 1024);
    B = B / (32 * NS) * (32 * NS);
    if (B < 32 * NS) B = 32 * NS;
    const int64_t spb = B / (32 * NS);   // slices per block
    const int64_t grid = (nslices + spb - 1) / spb;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(B);
    cfg.dynamicSmemBytes = (size_t)CW * B * 4;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (carveout >= 0) {
        attr[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
        attr[0].val.sharedMemCarveout = (unsigned)carveout;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, spmm_sell_f32_kernel<KP, NS>, p);
}

template <int KP>
static cudaError_t launch_f32(const SpmmParams<float>& p, int64_t nslices, SpmmConfig c,
                              cudaStream_t st)
{
    if constexpr (KP >= 16) {
        if (c.split == 4) return launch_f32_split<KP, 4>(p, nslices, c.carveout, st);
        if (c.split == 2) return launch_f32_split<KP, 2>(p, nslices, c.carveout, st);
    }
    return launch_f32_split<KP, 1>(p, nslices, c.carveout, st);
}

template <typename T>
cudaError_t launch_spmm(const SellDev& S, const EllDev& F, int k, T* Y,
                        int64_t ldy, SpmmConfig cfg, cudaStream_t st, int sm_count)
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
    p.frec = F.rec;
    p.dld = F.dld;
    p.fld = F.ld;
    p.heavy = F.heavy;
    p.k = k;
    p.Y = Y;
    p.partials = static_cast<T*>(S.partials);
    const int KP = F.ld;
    if constexpr (sizeof(T) == 4) {
        switch (KP) {
#define ESPNMF_KP(v) case v: return launch_f32<v>(p, S.nslices, cfg, st);
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

template <int KP>
static cudaError_t setup_f32()
{
    cudaError_t e = cudaFuncSetAttribute(spmm_sell_f32_kernel<KP, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    if constexpr (KP >= 16) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spmm_sell_f32_kernel<KP, 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spmm_sell_f32_kernel<KP, 4>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    }
    return e;
}

cudaError_t setup_spmm()
{
    cudaError_t e = cudaFuncSetAttribute(spmm_sell_f64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
#define ESPNMF_SETUP(v) if (e == cudaSuccess) e = setup_f32<v>();
    ESPNMF_SETUP(4) ESPNMF_SETUP(8) ESPNMF_SETUP(12) ESPNMF_SETUP(16)
    ESPNMF_SETUP(20) ESPNMF_SETUP(24) ESPNMF_SETUP(28) ESPNMF_SETUP(32)
    ESPNMF_SETUP(36) ESPNMF_SETUP(40) ESPNMF_SETUP(44) ESPNMF_SETUP(48)
    ESPNMF_SETUP(52) ESPNMF_SETUP(56) ESPNMF_SETUP(60) ESPNMF_SETUP(64)
    ESPNMF_SETUP(80) ESPNMF_SETUP(96) ESPNMF_SETUP(112) ESPNMF_SETUP(128)
#undef ESPNMF_SETUP
    return e;
}

template cudaError_t launch_spmm<float>(const SellDev&, const EllDev&, int, float*, int64_t, SpmmConfig, cudaStream_t, int);
template cudaError_t launch_spmm<double>(const SellDev&, const EllDev&, int, double*, int64_t, SpmmConfig, cudaStream_t, int);
template cudaError_t launch_spmm_combine<float>(const SellDev&, int, float*, int64_t, cudaStream_t);
template cudaError_t launch_spmm_combine<double>(const SellDev&, int, double*, int64_t, cudaStream_t);

}  // namespace espnmf
