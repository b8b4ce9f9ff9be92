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
//     almost every column's top-t) from the row's dense copy, in one of two
//     shapes:
//       lane-private: each lane reads its own entry's whole row (16-byte
//         loads) into KP register accumulators;
//       lane groups (k <= 64): the eight lanes of a group read each of the
//         group's heavy rows together, lane j taking chunks j and j + 8, so
//         a load instruction reads whole 128-byte lines; the group keeps the
//         heavy sums of its eight segments spread over its lanes by column
//         and moves them to their own lanes through shared memory once,
//         after the loop.
//     Lanes that each read 16 bytes of a different row are served at about
//     one line per cycle by the L1, lane groups at up to a line per cycle
//     per group; which shape wins depends on how many heavy rows stay in
//     the L1 (its share of the SM's memory is the launch's carveout), so the
//     host times both (SpmmConfig).  The shapes add the same products in the
//     same order: the result does not depend on the choice.
// The loop is software-pipelined: while a step's gathers run, the next
// step's records and the step after's entries of A are already in flight.
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

// FP32.  Light rows by their records into shared-memory slots (both modes);
// heavy rows either lane-private into KP register accumulators (GROUP =
// false) or by lane groups into column-distributed registers (GROUP = true,
// k <= 64).  The two modes add the same products in the same order, so they
// give bitwise the same Y.
template <int KP>
struct V4Shape {
    static constexpr int NCH = KP / 4;                 // 16-byte chunks of a row
    static constexpr int NC2 = NCH > 8 ? NCH - 8 : 0;  // lanes j < NC2 take a second chunk
    // heavy staging row stride: an odd number of chunks keeps the 128-bit
    // reads of eight consecutive segments' rows on distinct banks
    static constexpr int KPH = (NCH % 2 == 0) ? KP + 4 : KP;
};

template <int KP, bool GROUP>
__global__ void __launch_bounds__(256, KP <= 64 ? 2 : 1)
spmm_sell_f32_kernel(SpmmParams<float> p)
{
    using S = V4Shape<KP>;
    static_assert(!GROUP || KP <= 64, "lane groups cover at most 16 chunks");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NL = GROUP ? 8 : 1;      // heavy accumulator rows per lane
    constexpr int NA = GROUP ? 8 : KP;     // heavy accumulators per row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    float* slots = reinterpret_cast<float*>(smem_raw);                   // KP x B
    const int64_t s = (int64_t)blockIdx.x * (B >> 5) + warp;
    if (s >= p.nslices) return;
    const int64_t seg = s * 32 + lane;
    const int j = lane & 7;           // position in the lane group
    const int gb = lane & 24;         // first lane of the group

    float hacc[NL][NA];
#pragma unroll
    for (int L = 0; L < NL; ++L)
#pragma unroll
        for (int e = 0; e < NA; ++e) hacc[L][e] = 0.f;
    float* my = slots + tid;
#pragma unroll 4
    for (int c = 0; c < KP; ++c) my[c * B] = 0.f;

    const int len = p.slice_len[s];
    const int64_t base = p.slice_ptr[s] + lane;
    const int32_t* __restrict__ idx = p.idx + base;
    const float* __restrict__ val = p.val + base;
    const uint4* __restrict__ rec = p.frec;
    const float4* __restrict__ dense4 = reinterpret_cast<const float4*>(p.fdense);
    const int dld4 = p.dld / 4;
    const int heavy = p.heavy;
    const int fld = p.fld;
    bool any_heavy = false;

    auto light = [&](int i, float a, const uint4& r) {
        const int cnt = record_cnt(r.x);
        if (cnt == 0 || cnt >= heavy) return;
        my[((r.x >> 8) & 0xffu) * B] += a * __uint_as_float(r.y);
        if (cnt > 1) my[((r.x >> 16) & 0xffu) * B] += a * __uint_as_float(r.z);
        if (cnt > 2) my[(r.x >> 24) * B] += a * __uint_as_float(r.w);
        if (cnt > 3) {
            const int32_t* cr = p.fcol + (int64_t)i * fld;
            const float* vr = p.fval + (int64_t)i * fld;
            my[__ldg(cr + 3) * B] += a * __ldg(vr + 3);
            for (int q = 4; q < cnt; q += 4) {
                const int4 cc = __ldg(reinterpret_cast<const int4*>(cr + q));
                const float4 vv = __ldg(reinterpret_cast<const float4*>(vr + q));
                my[cc.x * B] += a * vv.x;
                if (q + 1 < cnt) my[cc.y * B] += a * vv.y;
                if (q + 2 < cnt) my[cc.z * B] += a * vv.z;
                if (q + 3 < cnt) my[cc.w * B] += a * vv.w;
            }
        }
    };
    // lane-private: this lane's heavy entry, its whole dense row
    auto heavy_lane = [&](int i, float a, bool h) {
        if (!h) return;
        const float4* r = dense4 + (int64_t)i * dld4;
#pragma unroll
        for (int q = 0; q < KP / 4; ++q) {
            const float4 v = __ldg(r + q);
            hacc[0][(4 * q + 0) % NA] = fmaf(a, v.x, hacc[0][(4 * q + 0) % NA]);
            hacc[0][(4 * q + 1) % NA] = fmaf(a, v.y, hacc[0][(4 * q + 1) % NA]);
            hacc[0][(4 * q + 2) % NA] = fmaf(a, v.z, hacc[0][(4 * q + 2) % NA]);
            hacc[0][(4 * q + 3) % NA] = fmaf(a, v.w, hacc[0][(4 * q + 3) % NA]);
        }
    };
    // lane groups: the heavy entries of two steps; group g gathers, for each
    // of its eight segments L, the dense rows of that segment's entries
    auto heavy_group = [&](int i0, float a0, bool h0, int i1, float a1, bool h1) {
        const unsigned m0 = __ballot_sync(FULL, h0);
        const unsigned m1 = __ballot_sync(FULL, h1);
        if ((m0 | m1) == 0u) return;
        any_heavy = true;
#pragma unroll
        for (int L = 0; L < NL; ++L) {
            const unsigned any0 = (m0 >> L) & 0x01010101u, any1 = (m1 >> L) & 0x01010101u;
            if ((any0 | any1) == 0u) continue;
            const int src = gb | L;
            const int r0 = __shfl_sync(FULL, i0, src);
            const float c0 = __shfl_sync(FULL, a0, src);
            const int r1 = __shfl_sync(FULL, i1, src);
            const float c1 = __shfl_sync(FULL, a1, src);
            const bool g0 = (m0 >> src) & 1u, g1 = (m1 >> src) & 1u;
            float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), y0 = x0, x1 = x0, y1 = x0;
            if (g0 && j < S::NCH) x0 = __ldg(dense4 + (int64_t)r0 * dld4 + j);
            if (g0 && j < S::NC2) y0 = __ldg(dense4 + (int64_t)r0 * dld4 + 8 + j);
            if (g1 && j < S::NCH) x1 = __ldg(dense4 + (int64_t)r1 * dld4 + j);
            if (g1 && j < S::NC2) y1 = __ldg(dense4 + (int64_t)r1 * dld4 + 8 + j);
            const float f0 = g0 ? c0 : 0.f, f1 = g1 ? c1 : 0.f;
            float* h = hacc[L];
            h[0 % NA] = fmaf(f1, x1.x, fmaf(f0, x0.x, h[0 % NA]));
            h[1 % NA] = fmaf(f1, x1.y, fmaf(f0, x0.y, h[1 % NA]));
            h[2 % NA] = fmaf(f1, x1.z, fmaf(f0, x0.z, h[2 % NA]));
            h[3 % NA] = fmaf(f1, x1.w, fmaf(f0, x0.w, h[3 % NA]));
            if (S::NC2 > 0) {
                h[4 % NA] = fmaf(f1, y1.x, fmaf(f0, y0.x, h[4 % NA]));
                h[5 % NA] = fmaf(f1, y1.y, fmaf(f0, y0.y, h[5 % NA]));
                h[6 % NA] = fmaf(f1, y1.z, fmaf(f0, y0.z, h[6 % NA]));
                h[7 % NA] = fmaf(f1, y1.w, fmaf(f0, y0.w, h[7 % NA]));
            }
        }
    };
    auto load2 = [&](int pp, int& i0, float& a0, int& i1, float& a1) {
        i0 = pp < len ? __ldcs(idx + (int64_t)pp * 32) : -1;
        a0 = pp < len ? __ldcs(val + (int64_t)pp * 32) : 0.f;
        i1 = pp + 1 < len ? __ldcs(idx + (int64_t)(pp + 1) * 32) : -1;
        a1 = pp + 1 < len ? __ldcs(val + (int64_t)(pp + 1) * 32) : 0.f;
    };
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);

    // stage j: entries (j, j+1) gathered; stage j+2's records and j+4's
    // entries are loaded meanwhile
    int i0, i1, n0, n1;
    float a0, a1, b0, b1;
    load2(0, i0, a0, i1, a1);
    load2(2, n0, b0, n1, b1);
    uint4 r0 = i0 >= 0 ? __ldg(rec + i0) : zero4;
    uint4 r1 = i1 >= 0 ? __ldg(rec + i1) : zero4;
    for (int p0 = 0; p0 < len; p0 += 2) {
        const uint4 q0 = n0 >= 0 ? __ldg(rec + n0) : zero4;
        const uint4 q1 = n1 >= 0 ? __ldg(rec + n1) : zero4;
        int m0, m1;
        float e0, e1;
        load2(p0 + 4, m0, e0, m1, e1);
        const bool h0 = record_cnt(r0.x) >= heavy, h1 = record_cnt(r1.x) >= heavy;
        light(i0, a0, r0);
        light(i1, a1, r1);
        if constexpr (GROUP) {
            heavy_group(i0, a0, h0, i1, a1, h1);
        } else {
            heavy_lane(i0, a0, h0);
            heavy_lane(i1, a1, h1);
        }
        i0 = n0; i1 = n1; a0 = b0; a1 = b1; r0 = q0; r1 = q1;
        n0 = m0; n1 = m1; b0 = e0; b1 = e1;
    }

    float acc[KP];
    if constexpr (GROUP) {
        if (__any_sync(FULL, any_heavy)) {
            // group g's column-distributed sums -> H[segment][column]; each
            // group writes whole 128-byte runs of one segment's row
            float* H = slots + (size_t)KP * B + (size_t)warp * 32 * S::KPH;
#pragma unroll
            for (int L = 0; L < NL; ++L) {
                float* hr = H + (gb | L) * S::KPH;
                if (j < S::NCH)
                    *reinterpret_cast<float4*>(hr + 4 * j) =
                        make_float4(hacc[L][0], hacc[L][1 % NA], hacc[L][2 % NA], hacc[L][3 % NA]);
                if (j < S::NC2)
                    *reinterpret_cast<float4*>(hr + 32 + 4 * j) =
                        make_float4(hacc[L][4 % NA], hacc[L][5 % NA], hacc[L][6 % NA], hacc[L][7 % NA]);
            }
            __syncwarp();
            const float* mine = H + lane * S::KPH;
#pragma unroll
            for (int q = 0; q < S::NCH; ++q) {
                const float4 h = *reinterpret_cast<const float4*>(mine + 4 * q);
                acc[4 * q + 0] = h.x + my[(4 * q + 0) * B];
                acc[4 * q + 1] = h.y + my[(4 * q + 1) * B];
                acc[4 * q + 2] = h.z + my[(4 * q + 2) * B];
                acc[4 * q + 3] = h.w + my[(4 * q + 3) * B];
            }
        } else {
#pragma unroll
            for (int c = 0; c < KP; ++c) acc[c] = my[c * B];
        }
    } else {
#pragma unroll
        for (int c = 0; c < KP; ++c) acc[c] = hacc[0][c % NA] + my[c * B];
    }
    // combine the lanes [head, end) of each row: fixed tree, lane head
    // ends with the row's sum
    const int grp = p.seg_grp[seg];
    const int head = grp >> 8, end = grp & 0xff;
    const int maxg = __reduce_max_sync(FULL, (unsigned)(end - head));
    for (int off = 1; off < maxg; off <<= 1) {
        const bool take = lane + off < end;
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            const float v = __shfl_down_sync(FULL, acc[c], off);
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

template <int KP, bool GROUP>
static cudaError_t launch_f32_mode(const SpmmParams<float>& p, int64_t nslices, int carveout,
                                   cudaStream_t st)
{
    const int B = spmm_block(KP, 4, 48 * 1024);
    const int64_t wpb = B / 32;
    const int64_t grid = (nslices + wpb - 1) / wpb;
    // slots (plus, for lane groups, the per-warp heavy staging rows)
    const size_t smem = (size_t)KP * B * 4 + (GROUP ? (size_t)B * V4Shape<KP>::KPH * 4 : 0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(B);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (carveout >= 0) {
        attr[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
        attr[0].val.sharedMemCarveout = (unsigned)carveout;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, spmm_sell_f32_kernel<KP, GROUP>, p);
}

template <int KP>
static cudaError_t launch_f32(const SpmmParams<float>& p, int64_t nslices, SpmmConfig c,
                              cudaStream_t st)
{
    if constexpr (KP <= 64) {
        if (c.group) return launch_f32_mode<KP, true>(p, nslices, c.carveout, st);
    }
    return launch_f32_mode<KP, false>(p, nslices, c.carveout, st);
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
    cudaError_t e = cudaFuncSetAttribute(spmm_sell_f32_kernel<KP, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    if constexpr (KP <= 64) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spmm_sell_f32_kernel<KP, true>,
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
