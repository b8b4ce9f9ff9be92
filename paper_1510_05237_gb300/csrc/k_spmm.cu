// k_spmm.cu -- the sparse products of Alg. 2 steps 1 and 3:
//   Y = A^T U (V half)   and   Y = A V (U half).
//
// Each product has up to two parts, run one after the other on the stream.
//
// SELL part (spmm_sell_*): A's entries are streamed once from a
// sliced-ELLPACK layout (SELL-32): a warp's 32 lanes walk 32 segments of
// about the same length, so every load of A is a coalesced 128-byte
// transaction.  A row is cut into 1..32 segments of at most 64 entries held
// by adjacent lanes; each lane sums its segment and the lanes of a row are
// combined by a fixed shuffle tree.  The factor row an entry gathers is read
// sparsely: a bitmask (L1-resident or in shared memory) skips rows that are
// zero; otherwise the row's 32-byte record (one L2 sector) holds its count
// and first six (column, value) pairs -- the first 16-byte half the first
// three -- longer rows continue in the row-packed pairs, and the rare dense
// row is read from its dense copy.  Every product is added into per-thread
// accumulators in shared memory, slot c of thread tid at acc[c * B + tid]
// (a warp's lanes always touch 32 distinct banks, whatever columns they
// update), so a thread needs few registers and many warps stay resident to
// hide the latency of the gathers.
//
// Frequent part (spmm_freq_f32, FP32 form): on text corpora the factor rows
// of the most frequent terms end up in nearly every column's top t, so the
// entries that gather them (a large share of A's nonzeros) would each cost
// a dense row of scattered loads.  These h rows are chosen once, when the
// context is built (the gathered rows that the most entries of A reference,
// as many as fit a 200 KB table); their entries are stored apart from the
// SELL arrays, per output row, as (table row offset, value) with each row
// padded to a multiple of the warp's step.  One persistent CTA per SM stages
// the dense copies of the h rows in shared memory with a TMA bulk copy; each
// warp streams a chunk of rows' entries through a ring in shared memory
// (cp.async, two stages ahead), a group of lanes per entry reading the
// entry's table row with 128-bit shared loads (lanes over columns,
// conflict-free), and adds each row's sum into the row of Y that the SELL
// part wrote.
//
// All sums are taken in a fixed order (storage order per lane, a fixed tree
// across lanes, chunk order for very long rows, a fixed entry order per
// group of lanes and a fixed tree across groups), so the product is bitwise
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
    const uint32_t* fmask;
    int mask_words;   // words of fmask (staged in shared memory when MASK == 2)
    int dld;
    int fld;
    int64_t frows;   // rows of the gathered factor
    int64_t yrows;   // output rows
    int64_t npart;   // partial rows
    int heavy;
    int k;
    T* Y;        // rows x KP (ldy == KP)
    T* partials; // npart x KP
};

// End of a slice: combines the lanes [head, end) of each row, four columns
// at a time (a fixed tree; lane head ends with the row's sum), and writes
// columns [c0, c0 + cw) of the row of Y, or of its partial row.
template <int KP>
__device__ __forceinline__ void sell_store_rows(const SpmmParams<float>& p, int64_t seg, int lane,
                                                const float* my, int B, int c0, int cw)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int grp = p.seg_grp[seg];
    const int head = grp >> 8, end = grp & 0xff;
    const int maxg = __reduce_max_sync(FULL, (unsigned)(end - head));
    const int row = p.seg_row[seg];
    const int part = p.seg_part[seg];
    const bool in_range = row < 0 || ESPNMF_CHECK(part < 0 ? row < p.yrows : part < p.npart, CHK_OUT_ROW);
    float* out = (part < 0 ? p.Y + (int64_t)(row < 0 || !in_range ? 0 : row) * KP
                           : p.partials + (int64_t)(in_range ? part : 0) * KP) + c0;
    float4* o4 = reinterpret_cast<float4*>(out);
    const bool writer = row >= 0 && in_range && lane == head;
#pragma unroll 1
    for (int q = 0; 4 * q < cw; ++q) {
        float v0 = my[(4 * q + 0) * B], v1 = my[(4 * q + 1) * B];
        float v2 = my[(4 * q + 2) * B], v3 = my[(4 * q + 3) * B];
        for (int off = 1; off < maxg; off <<= 1) {
            const bool take = lane + off < end;
            const float t0 = __shfl_down_sync(FULL, v0, off);
            const float t1 = __shfl_down_sync(FULL, v1, off);
            const float t2 = __shfl_down_sync(FULL, v2, off);
            const float t3 = __shfl_down_sync(FULL, v3, off);
            if (take) {
                v0 += t0;
                v1 += t1;
                v2 += t2;
                v3 += t3;
            }
        }
        if (writer) o4[q] = make_float4(v0, v1, v2, v3);
    }
}

// FP32.  NS warps share a slice: warp h of the NS owns the output columns
// [h * CW, min(KP, (h + 1) * CW)), CW = KP / NS rounded up to 4, for all 32
// segments of the slice.  Each of them streams the slice's entries (the NS
// warps read the same lines, mostly from L1) and adds the products for its
// columns into its slots.  A larger NS means fewer slots per thread, so more
// warps in flight for the same shared memory, at the price of re-reading A
// and the records.  Every NS adds the same products in the same order.
template <int KP, int NS>
struct SplitShape {
    static constexpr int CW = ((KP + NS - 1) / NS + 3) / 4 * 4;
};

// MASK: 0 -- every entry loads its row's record; 1 -- zero rows are skipped
// by the bitmask in global memory (the L1/L2); 2 -- the bitmask is first
// copied into shared memory (after the slots).
template <int KP, int NS, int MASK>
__global__ void __launch_bounds__(256, 4)
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
    const uint32_t* __restrict__ fmask = p.fmask;
    if constexpr (MASK == 2) {
        uint32_t* sm = reinterpret_cast<uint32_t*>(slots + (size_t)CW * B);
        for (int w = tid; w < p.mask_words; w += B) sm[w] = __ldg(p.fmask + w);
        __syncthreads();
        fmask = sm;
    }
    if (cw <= 0) return;
    float* my = slots + tid;
    const uint4* __restrict__ rec = p.frec;
    const float4* __restrict__ dense4 = reinterpret_cast<const float4*>(p.fdense) + c0 / 4;
    const int dld4 = p.dld / 4;
    const int heavy = p.heavy;
    const int fld = p.fld;
    const unsigned ucw = (unsigned)cw;

    // one product of a row's pair: column c (absolute) if this warp owns it.
    // Every accumulation is an explicit fused multiply-add, so that all
    // launch shapes (different instantiations) round the same way.
    auto add = [&](unsigned c, float a, float v) {
        const unsigned r = c - (unsigned)c0;
        if (r < ucw && ESPNMF_CHECK(c < (unsigned)KP, CHK_COLUMN)) my[r * B] = __fmaf_rn(a, v, my[r * B]);
    };
    // the pairs of row i beyond the record's three, or the whole dense copy
    // of a heavy row
    auto gather_long = [&](int i, float a, int cnt) {
        if (!ESPNMF_CHECK(cnt <= fld, CHK_COUNT)) return;
        if (cnt >= heavy) {
            const float4* d = dense4 + (int64_t)i * dld4;
            for (int q = 0; 4 * q < cw; ++q) {
                const float4 v = __ldg(d + q);
                my[(4 * q + 0) * B] = __fmaf_rn(a, v.x, my[(4 * q + 0) * B]);
                my[(4 * q + 1) * B] = __fmaf_rn(a, v.y, my[(4 * q + 1) * B]);
                my[(4 * q + 2) * B] = __fmaf_rn(a, v.z, my[(4 * q + 2) * B]);
                my[(4 * q + 3) * B] = __fmaf_rn(a, v.w, my[(4 * q + 3) * B]);
            }
            return;
        }
        const int32_t* cr = p.fcol + (int64_t)i * fld;
        const float* vr = p.fval + (int64_t)i * fld;
        add((unsigned)__ldg(cr + 3), a, __ldg(vr + 3));
        for (int q = 4; q < cnt; q += 4) {
            const int4 cc = __ldg(reinterpret_cast<const int4*>(cr + q));
            const float4 vv = __ldg(reinterpret_cast<const float4*>(vr + q));
            add((unsigned)cc.x, a, vv.x);
            if (q + 1 < cnt) add((unsigned)cc.y, a, vv.y);
            if (q + 2 < cnt) add((unsigned)cc.z, a, vv.z);
            if (q + 3 < cnt) add((unsigned)cc.w, a, vv.w);
        }
    };
    // Slices are sorted longest first; the warps (groups of NS) take them
    // round-robin, so every warp gets about the same work.
    const int64_t stride = (int64_t)gridDim.x * (B >> 5) / NS;
    for (int64_t s = (int64_t)blockIdx.x * (B >> 5) / NS + warp / NS; s < p.nslices; s += stride) {
        const int64_t seg = s * 32 + lane;
#pragma unroll 4
        for (int c = 0; c < CW; ++c) my[c * B] = 0.f;
        const int len = p.slice_len[s];   // a multiple of 4
        const int nq = len >> 2;
        const int64_t base = p.slice_ptr[s] + lane * 4;
        const int4* __restrict__ idx4 = reinterpret_cast<const int4*>(p.idx + base);
        const float4* __restrict__ val4 = reinterpret_cast<const float4*>(p.val + base);

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

        // Quads of four entries per lane (one 16-byte load of indices and
        // one of values), two quads ahead.  A quad's bitmask words (MASK),
        // then its records, are loaded together (four independent loads per
        // stage).  Its products: the record's pairs (up to three per entry)
        // as twelve pair slots, visited in order and only where some lane
        // of the warp has a pair, so the warp does not diverge; rows with
        // more nonzeros (rare in an enforced-sparse factor) afterwards.
        const int4 none_i = make_int4(-1, -1, -1, -1);
        const float4 none_a = make_float4(0.f, 0.f, 0.f, 0.f);
        const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
        int4 i0 = nq > 0 ? __ldcs(idx4) : none_i;
        float4 a0 = nq > 0 ? __ldcs(val4) : none_a;
        int4 i1 = nq > 1 ? __ldcs(idx4 + 32) : none_i;
        float4 a1 = nq > 1 ? __ldcs(val4 + 32) : none_a;
        for (int q = 0; q < nq; ++q) {
            int4 i2 = none_i;
            float4 a2 = none_a;
            if (q + 2 < nq) {
                i2 = __ldcs(idx4 + (int64_t)(q + 2) * 32);
                a2 = __ldcs(val4 + (int64_t)(q + 2) * 32);
            }
            int ii[4] = {i0.x, i0.y, i0.z, i0.w};
            const float aa[4] = {a0.x, a0.y, a0.z, a0.w};
            uint4 rc[4];
            if constexpr (MASK > 0) {
                // skip the records of zero rows (one more dependent load)
                uint32_t mw[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (ii[u] >= 0 && !ESPNMF_CHECK(ii[u] < p.frows, CHK_FACTOR_ROW)) ii[u] = -1;
#pragma unroll
                for (int u = 0; u < 4; ++u) mw[u] = ii[u] >= 0 ? fmask[ii[u] >> 5] : 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    rc[u] = (ii[u] >= 0 && ((mw[u] >> (ii[u] & 31)) & 1u)) ? __ldg(rec + 2 * ii[u]) : zero4;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (ii[u] >= 0 && !ESPNMF_CHECK(ii[u] < p.frows, CHK_FACTOR_ROW)) ii[u] = -1;
#pragma unroll
                for (int u = 0; u < 4; ++u) rc[u] = ii[u] >= 0 ? __ldg(rec + 2 * ii[u]) : zero4;
            }
            // this lane's pair slots (bit 3u + j: pair j of entry u) and its
            // longer rows (bit 12 + u)
            unsigned mine = 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = record_cnt(rc[u].x);
                const int light = c >= heavy ? 0 : (c < 3 ? c : 3);
                mine |= ((1u << light) - 1u) << (3 * u);
                if (c > 3) mine |= 1u << (12 + u);
            }
            const unsigned need = __reduce_or_sync(FULL, mine);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const unsigned bit = 1u << (3 * u + j);
                    if (need & bit) {
                        if (mine & bit) {
                            const unsigned col = (rc[u].x >> (8 * (j + 1))) & 0xffu;
                            const unsigned vb = j == 0 ? rc[u].y : (j == 1 ? rc[u].z : rc[u].w);
                            add(col, aa[u], __uint_as_float(vb));
                        }
                    }
                }
            }
            if (need >> 12) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (mine & (1u << (12 + u))) gather_long(ii[u], aa[u], record_cnt(rc[u].x));
            }
            i0 = i1;
            a0 = a1;
            i1 = i2;
            a1 = a2;
        }

        sell_store_rows<KP>(p, seg, lane, my, B, c0, cw);
    }
}

// FP32, one warp per slice (all columns), the shape the tuner picks on text
// corpora.  The same products as spmm_sell_f32_kernel<KP, 1, MASK>, added
// in the same order, with fewer instructions and fewer dependent loads per
// entry.  A record's unused pair slots hold column 0 and value +0, so pair 0
// of every entry is added without a branch (a zero row, a padding entry or
// a heavy row adds +0 into slot 0, which leaves it unchanged: every product
// is >= 0, so no slot is ever -0).  Pairs 1 and 2 of entry u are added only
// when some lane of the warp has a light row with two or more nonzeros
// there (a warp-uniform branch; one reduction per quad gives all of them).
// Pairs 3 to 5 come from the record's second half, which shares the first
// half's 32-byte sector (an L1 hit), not from the row-packed pairs in the
// L2; only rows of more than six nonzeros read those, and heavy rows their
// dense copy.  The four entries of a quad are held in plain registers and a
// slot's address is one multiply-add from its column.
template <int KP, int MASK>
__global__ void __launch_bounds__(256, 4)
spmm_sell1_f32_kernel(SpmmParams<float> p)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    float* slots = reinterpret_cast<float*>(smem_raw);                   // KP x B
    const uint32_t* __restrict__ fmask = p.fmask;
    if constexpr (MASK == 2) {
        uint32_t* sm = reinterpret_cast<uint32_t*>(slots + (size_t)KP * B);
        for (int w = tid; w < p.mask_words; w += B) sm[w] = __ldg(p.fmask + w);
        __syncthreads();
        fmask = sm;
    }
    float* my = slots + tid;
    const unsigned bstride = (unsigned)B * 4u;                // bytes between a thread's slots
    const uint32_t mybase = (uint32_t)__cvta_generic_to_shared(my);
    const uint4* __restrict__ rec = p.frec;
    const float4* __restrict__ dense4 = reinterpret_cast<const float4*>(p.fdense);
    const int dld4 = p.dld / 4;
    const int heavy = p.heavy;
    const int fld = p.fld;

    // slot[col] += a * v (an explicit fused multiply-add, as in every shape)
    auto fma_slot = [&](unsigned col, float a, float v) {
        if (!ESPNMF_CHECK(col < (unsigned)KP, CHK_COLUMN)) return;
        const uint32_t ad = mybase + col * bstride;
        float s;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(s) : "r"(ad));
        s = __fmaf_rn(a, v, s);
        asm volatile("st.shared.f32 [%0], %1;" :: "r"(ad), "f"(s) : "memory");
    };
    // pairs 3.. of row i (cnt of them in all): 3 to 5 from the record's
    // second half, the rest from the row-packed pairs; a heavy row from its
    // dense copy
    auto pairs_beyond = [&](int i, float a, int cnt) {
        if (!ESPNMF_CHECK(cnt <= fld, CHK_COUNT)) return;
        if (cnt >= heavy) {
            const float4* d = dense4 + (int64_t)i * dld4;
#pragma unroll 1
            for (int q = 0; 4 * q < KP; ++q) {
                const float4 v = __ldg(d + q);
                my[(4 * q + 0) * B] = __fmaf_rn(a, v.x, my[(4 * q + 0) * B]);
                my[(4 * q + 1) * B] = __fmaf_rn(a, v.y, my[(4 * q + 1) * B]);
                my[(4 * q + 2) * B] = __fmaf_rn(a, v.z, my[(4 * q + 2) * B]);
                my[(4 * q + 3) * B] = __fmaf_rn(a, v.w, my[(4 * q + 3) * B]);
            }
            return;
        }
        const uint4 h = __ldg(rec + 2 * i + 1);
        fma_slot(__byte_perm(h.x, 0u, 0x4440), a, __uint_as_float(h.y));
        if (cnt > 4) fma_slot(__byte_perm(h.x, 0u, 0x4441), a, __uint_as_float(h.z));
        if (cnt > 5) fma_slot(__byte_perm(h.x, 0u, 0x4442), a, __uint_as_float(h.w));
        if (cnt > 6) {
            const int32_t* cr = p.fcol + (int64_t)i * fld;
            const float* vr = p.fval + (int64_t)i * fld;
#pragma unroll 1
            for (int q = 6; q < cnt; ++q) fma_slot((unsigned)__ldg(cr + q), a, __ldg(vr + q));
        }
    };
    // the first half of row i's record (zero for a padding entry or, with
    // the bitmask, a zero row)
    auto load_rec = [&](int i) -> uint4 {
        bool live = i >= 0 && ESPNMF_CHECK(i < p.frows, CHK_FACTOR_ROW);
        if constexpr (MASK > 0) live = live && ((fmask[i >> 5] >> (i & 31)) & 1u);
        return live ? __ldg(rec + 2 * i) : make_uint4(0u, 0u, 0u, 0u);
    };
    // pair 0 of an entry, then (warp-uniform) its pairs 1 and 2
    auto light_pairs = [&](const uint4& r, float a, bool more) {
        const bool lt = record_cnt(r.x) < heavy;
        fma_slot(__byte_perm(r.x, 0u, 0x4441), a, lt ? __uint_as_float(r.y) : 0.f);
        if (more) {
            fma_slot(__byte_perm(r.x, 0u, 0x4442), a, lt ? __uint_as_float(r.z) : 0.f);
            fma_slot(__byte_perm(r.x, 0u, 0x4443), a, lt ? __uint_as_float(r.w) : 0.f);
        }
    };

    const int64_t stride = (int64_t)gridDim.x * (B >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (B >> 5) + warp; s < p.nslices; s += stride) {
        const int64_t seg = s * 32 + lane;
#pragma unroll 4
        for (int c = 0; c < KP; ++c) my[c * B] = 0.f;
        const int len = p.slice_len[s];   // a multiple of 4
        const int nq = len >> 2;
        const int64_t base = p.slice_ptr[s] + lane * 4;
        const int4* __restrict__ idx4 = reinterpret_cast<const int4*>(p.idx + base);
        const float4* __restrict__ val4 = reinterpret_cast<const float4*>(p.val + base);
        if (lane == 0 && len > 0) {
            const unsigned bytes = (unsigned)len * 128u;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         :: "l"(p.idx + p.slice_ptr[s]), "r"(bytes) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         :: "l"(p.val + p.slice_ptr[s]), "r"(bytes) : "memory");
        }
        const int4 none_i = make_int4(-1, -1, -1, -1);
        const float4 none_a = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 i0 = nq > 0 ? __ldcs(idx4) : none_i;
        float4 a0 = nq > 0 ? __ldcs(val4) : none_a;
        int4 i1 = nq > 1 ? __ldcs(idx4 + 32) : none_i;
        float4 a1 = nq > 1 ? __ldcs(val4 + 32) : none_a;
#pragma unroll 1
        for (int q = 0; q < nq; ++q) {
            int4 i2 = none_i;
            float4 a2 = none_a;
            if (q + 2 < nq) {
                i2 = __ldcs(idx4 + (int64_t)(q + 2) * 32);
                a2 = __ldcs(val4 + (int64_t)(q + 2) * 32);
            }
            const uint4 r0 = load_rec(i0.x), r1 = load_rec(i0.y);
            const uint4 r2 = load_rec(i0.z), r3 = load_rec(i0.w);
            // byte u of `need`: the OR over the warp of entry u's count, so
            // >= 2 iff some lane's row has two or more nonzeros there and
            // >= 4 iff some lane's has more than three (heavy rows included:
            // their pairs 1 and 2 add +0)
            const unsigned need = __reduce_or_sync(
                FULL, __byte_perm(__byte_perm(r0.x, r1.x, 0x0040), __byte_perm(r2.x, r3.x, 0x0040), 0x5410));
            light_pairs(r0, a0.x, (need & 0xffu) >= 2u);
            light_pairs(r1, a0.y, ((need >> 8) & 0xffu) >= 2u);
            light_pairs(r2, a0.z, ((need >> 16) & 0xffu) >= 2u);
            light_pairs(r3, a0.w, (need >> 24) >= 2u);
            if ((need & 0xfcfcfcfcu) != 0u) {
                if (record_cnt(r0.x) > 3) pairs_beyond(i0.x, a0.x, record_cnt(r0.x));
                if (record_cnt(r1.x) > 3) pairs_beyond(i0.y, a0.y, record_cnt(r1.x));
                if (record_cnt(r2.x) > 3) pairs_beyond(i0.z, a0.z, record_cnt(r2.x));
                if (record_cnt(r3.x) > 3) pairs_beyond(i0.w, a0.w, record_cnt(r3.x));
            }
            i0 = i1;
            a0 = a1;
            i1 = i2;
            a1 = a2;
        }
        sell_store_rows<KP>(p, seg, lane, my, B, 0, KP);
    }
}

// ---------------------------------------------------------------------------
// Frequent part (FP32).

// A group of LPG lanes (a power of two, >= KP / 4, at least two) handles
// one entry: lane ql of the group holds the float4 of columns [4 ql, 4 ql +
// 4).  A warp step adds STEP = 2 G entries, two per group (G = 32 / LPG).
constexpr int freq_lanes(int kp)
{
    return kp / 4 <= 2 ? 2 : kp / 4 <= 4 ? 4 : kp / 4 <= 8 ? 8 : kp / 4 <= 16 ? 16 : 32;
}
template <int KP>
struct FreqShape {
    static constexpr int Q = KP / 4;
    static constexpr int LPG = freq_lanes(KP);
    static constexpr int G = 32 / LPG;
    static constexpr int STEP = 2 * G;
};

int freq_pad(int ld)
{
    const int step = 2 * (32 / freq_lanes(ld));
    return step > 4 ? step : 4;
}

// the ring of entry stages of all warps of a CTA (32 entries of 8 bytes each)
constexpr uint32_t kFreqRingBytes = (uint32_t)(kHThreads / 32) * kFreqStages * 256u;

struct FreqParams {
    const uint2* ent;      // (table row byte offset, value bits), rows padded
    const int2* rows;      // (output row, end of its entries / 4)
    const int32_t* chunk;  // [nchunks + 1] ranges of rows
    int nchunks;
    int* counter;
    const float* htab;     // the factor's table [h_all + 1][KP] (row h_all zero)
    int h;                 // tier 1: rows staged (a zero row after them); tier 2: h_all
    float* Y;              // rows x KP: holds the SELL part, receives the sum
    unsigned* status;
    long long wait_limit;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Two FP32 lanes in one 64-bit register: (x, y) = (low, high) word.
__device__ __forceinline__ unsigned long long pack2(float a)
{
    const unsigned long long u = __float_as_uint(a);
    return u | (u << 32);
}
// acc = a * v + acc on both lanes (IEEE round-to-nearest fused multiply-add
// per lane, the same rounding as fmaf).
__device__ __forceinline__ void fma2(unsigned long long& acc, unsigned long long a,
                                     unsigned long long v)
{
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(v));
}
__device__ __forceinline__ float4 unpack4(unsigned long long xy, unsigned long long zw)
{
    return make_float4(__uint_as_float((unsigned)xy), __uint_as_float((unsigned)(xy >> 32)),
                       __uint_as_float((unsigned)zw), __uint_as_float((unsigned)(zw >> 32)));
}

// Waits (bounded) for phase 0 of the mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait_phase0(uint32_t mbar, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(0u) : "memory");
        if (done) return true;
    }
    return false;
}

// GLOBAL = false: the first tier, the table staged in shared memory (p.h
// rows and a zero row after them); GLOBAL = true: the second tier, table
// rows read from the factor's table in global memory (p.htab, p.h rows and
// its zero row h), which stays in the L2.
//
// A warp takes a chunk of rows and streams the chunk's entries (one
// contiguous run) through its ring of kFreqStages stages of 32 entries,
// filled by cp.async two stages ahead of the one being added.  Step by
// step, group g adds the entry pair (STEP i + 2 g, STEP i + 2 g + 1) of the
// row with packed two-lane FMAs (each lane rounds as fmaf does) into two
// accumulators; a zero table row adds +0.  Rows are padded to a multiple of
// the step, so a row ends at a step boundary: there the groups' sums are
// combined in a fixed tree and group 0 adds them to the row of Y.  Every
// row is summed by one warp in a fixed order, whichever warp takes it.
template <int KP, bool GLOBAL>
__global__ void __launch_bounds__(kHThreads, 1)
spmm_freq_f32_kernel(FreqParams p)
{
    using S = FreqShape<KP>;
    constexpr int Q = S::Q, LPG = S::LPG, STEP = S::STEP;
    constexpr int NST = kFreqStages;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr uint32_t ROW = KP * 4;   // bytes per table row
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    // the table and its zero row (tier 1), then the warps' rings
    const uint32_t tab_bytes = GLOBAL ? 0u : ((uint32_t)p.h + 1u) * ROW;
    const uint32_t ring = smem_addr(smem_raw) + tab_bytes + (uint32_t)warp * (NST * 256u);

    // stage the dense table: TMA bulk copies (32 KB each) completing on one
    // mbarrier; the zero row after it by plain stores meanwhile
    if constexpr (!GLOBAL) {
    float* tab = reinterpret_cast<float*>(smem_raw);   // [h + 1][KP], row h zero
    const uint32_t bar = smem_addr(&mbar);
    const uint32_t bytes = (uint32_t)p.h * ROW;   // a multiple of 16
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(bar), "r"(bytes) : "memory");
        for (uint32_t off = 0; off < bytes; off += 32768u) {
            const uint32_t n = bytes - off < 32768u ? bytes - off : 32768u;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                :: "r"(smem_addr(smem_raw + off)), "l"(reinterpret_cast<const unsigned char*>(p.htab) + off),
                   "r"(n), "r"(bar) : "memory");
        }
    }
    for (int c = tid; c < KP; c += blockDim.x) tab[(size_t)p.h * KP + c] = 0.f;
    __syncthreads();
    if (!mbar_wait_phase0(bar, p.wait_limit)) {
        // the copy did not land: report, give it one more bounded wait so
        // that it does not write into a later CTA's memory, and stop
        if (tid == 0) atomicOr(p.status, ST_TIMEOUT);
        mbar_wait_phase0(bar, p.wait_limit);
        return;
    }
    }

    const int grp = lane / LPG, ql = lane % LPG;
    const bool colact = ql < Q;
    const bool writer = grp == 0 && colact;
    const uint32_t zero_off = (uint32_t)p.h * ROW;
    const uint32_t lane_base = GLOBAL ? 0u : smem_addr(smem_raw) + 16u * (uint32_t)ql;
    const unsigned char* gbase = reinterpret_cast<const unsigned char*>(p.htab) + 16u * (uint32_t)ql;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // The warps take chunks in turn (a CTA that starts late, e.g. on an SM
    // shared with another kernel, does not hold the others up).
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(p.counter, 1);
        ch = __shfl_sync(FULL, ch, 0);
        if (ch >= p.nchunks) break;
        const int k0 = p.chunk[ch], k1 = p.chunk[ch + 1];
        if (k0 >= k1) continue;
        const int qa = k0 > 0 ? p.rows[k0 - 1].y : 0;   // the chunk's entries: 4 qa ..
        const int ne = 4 * (p.rows[k1 - 1].y - qa);     // .. 4 qa + ne
        const uint2* src = p.ent + 4ll * qa;
        if (lane == 0 && ne > 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         :: "l"(src), "r"((unsigned)ne * 8u) : "memory");
        // stage s holds the chunk's entries [32 s, 32 s + 32) in slot s % NST;
        // lanes 0..15 copy 16 bytes each.  Every lane commits a group per
        // stage (empty beyond the chunk), so waiting for all but the last
        // NST - 1 groups means stage s has landed.
        auto issue = [&](int st) {
            const int e = 32 * st + 2 * lane;
            if (lane < 16 && e < ne) {
                const uint32_t dst = ring + (uint32_t)(st % NST) * 256u + 16u * (uint32_t)lane;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                             :: "r"(dst), "l"(src + e) : "memory");
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        __syncwarp();   // the previous chunk's reads of the ring are done
#pragma unroll
        for (int st = 0; st < NST - 1; ++st) issue(st);
        int j = k0;                        // the row being summed
        int2 cur = p.rows[k0];
        int rend = 4 * (cur.y - qa);       // its end within the chunk
        int2 nxt = j + 1 < k1 ? p.rows[j + 1] : cur;
        float4* yr = reinterpret_cast<float4*>(p.Y + (int64_t)cur.x * KP) + ql;
        float4 yv = writer ? *yr : zero4;
        unsigned long long a0xy = 0ull, a0zw = 0ull, a1xy = 0ull, a1zw = 0ull;
        for (int st = 0; 32 * st < ne; ++st) {
            __syncwarp();   // stage st - 1 is read: its slot takes stage st + NST - 1
            issue(st + NST - 1);
            asm volatile("cp.async.wait_group %0;" :: "n"(NST - 1) : "memory");
            __syncwarp();   // every lane's copies of stage st have landed
            const uint32_t sb = ring + (uint32_t)(st % NST) * 256u + 16u * (uint32_t)grp;
            const int e0 = 32 * st;
            const int se = ne - e0 < 32 ? ne - e0 : 32;
            for (int jj = 0; jj < se; jj += STEP) {
                int4 ee;   // this group's entries jj + 2 grp, jj + 2 grp + 1
                asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(ee.x), "=r"(ee.y), "=r"(ee.z), "=r"(ee.w)
                             : "r"(sb + 8u * (uint32_t)jj));
                if (!ESPNMF_CHECK((uint32_t)ee.x <= zero_off && (uint32_t)ee.z <= zero_off &&
                                  (((uint32_t)ee.x | (uint32_t)ee.z) & 15u) == 0u, CHK_SLOT)) {
                    ee = make_int4((int)zero_off, 0, (int)zero_off, 0);
                }
                if (colact) {
                    unsigned long long v0x, v0y, v1x, v1y;
                    if constexpr (GLOBAL) {
                        asm volatile("ld.global.nc.v2.b64 {%0, %1}, [%2];"
                                     : "=l"(v0x), "=l"(v0y) : "l"(gbase + (uint32_t)ee.x));
                        asm volatile("ld.global.nc.v2.b64 {%0, %1}, [%2];"
                                     : "=l"(v1x), "=l"(v1y) : "l"(gbase + (uint32_t)ee.z));
                    } else {
                        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
                                     : "=l"(v0x), "=l"(v0y) : "r"(lane_base + (uint32_t)ee.x));
                        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
                                     : "=l"(v1x), "=l"(v1y) : "r"(lane_base + (uint32_t)ee.z));
                    }
                    const unsigned long long a0 = pack2(__int_as_float(ee.y));
                    const unsigned long long a1 = pack2(__int_as_float(ee.w));
                    fma2(a0xy, a0, v0x);
                    fma2(a0zw, a0, v0y);
                    fma2(a1xy, a1, v1x);
                    fma2(a1zw, a1, v1y);
                }
                if (e0 + jj + STEP == rend) {
                    // the row is complete: the groups' sums in a fixed tree,
                    // group 0 adds them to the SELL part
                    const float4 acc0 = unpack4(a0xy, a0zw), acc1 = unpack4(a1xy, a1zw);
                    float4 acc = make_float4(acc0.x + acc1.x, acc0.y + acc1.y,
                                             acc0.z + acc1.z, acc0.w + acc1.w);
#pragma unroll
                    for (int off = LPG; off < 32; off <<= 1) {
                        acc.x += __shfl_xor_sync(FULL, acc.x, off);
                        acc.y += __shfl_xor_sync(FULL, acc.y, off);
                        acc.z += __shfl_xor_sync(FULL, acc.z, off);
                        acc.w += __shfl_xor_sync(FULL, acc.w, off);
                    }
                    if (writer)
                        *yr = make_float4(yv.x + acc.x, yv.y + acc.y, yv.z + acc.z, yv.w + acc.w);
                    a0xy = a0zw = a1xy = a1zw = 0ull;
                    if (++j < k1) {
                        cur = nxt;
                        rend = 4 * (cur.y - qa);
                        yr = reinterpret_cast<float4*>(p.Y + (int64_t)cur.x * KP) + ql;
                        yv = writer ? *yr : zero4;
                        if (j + 1 < k1) nxt = p.rows[j + 1];
                    }
                }
            }
        }
    }
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
    const int64_t base = p.slice_ptr[s] + lane * 4;
    const int heavy = p.heavy;
    for (int p0 = 0; p0 < len; ++p0) {
        const int64_t at = base + (int64_t)(p0 >> 2) * 128 + (p0 & 3);
        int i = __ldcs(p.idx + at);
        const double a = __ldcs(p.val + at);
        if (i >= 0 && !ESPNMF_CHECK(i < p.frows, CHK_FACTOR_ROW)) i = -1;
        int cnt = i >= 0 ? __ldg(p.fcnt + i) : 0;
        if (!ESPNMF_CHECK(cnt <= KP, CHK_COUNT)) cnt = 0;
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
                const bool ok = ESPNMF_CHECK((unsigned)cc.x < (unsigned)KP &&
                                                 (q + 1 >= cnt || (unsigned)cc.y < (unsigned)KP) &&
                                                 (q + 2 >= cnt || (unsigned)cc.z < (unsigned)KP) &&
                                                 (q + 3 >= cnt || (unsigned)cc.w < (unsigned)KP),
                                             CHK_COLUMN);
                if (!ok) continue;
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
    const bool in_range = row < 0 || ESPNMF_CHECK(part < 0 ? row < p.yrows : part < p.npart, CHK_OUT_ROW);
    double* out = (row >= 0 && in_range && lane == head)
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
        // eight partials loaded before they are added, in order
        for (int q0 = 0; q0 < count; q0 += 8) {
            T b[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) b[u] = q0 + u < count ? pp[(int64_t)(q0 + u) * KP] : T(0);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (q0 + u < count) s0 += b[u];
        }
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

// Resident blocks per SM of each FP32 SELL instantiation, found by the
// per-device set-up (before any capture) and read by the launches.
static int g_sell_per_sm[129][5][3];

template <int KP, int NS>
static int sell_block(int& B)
{
    constexpr int CW = SplitShape<KP, NS>::CW;
    // NS warps per slice; at most 56 KB of slots per block (four blocks of
    // 256 threads per SM at k = 50)
    B = spmm_block(CW, 4, 56 * 1024);
    B = B / (32 * NS) * (32 * NS);
    if (B < 32 * NS) B = 32 * NS;
    return CW * B * 4;
}

template <int KP, int NS, int MASK>
static cudaError_t launch_f32_split(const SpmmParams<float>& p, int64_t nslices, int carveout,
                                    cudaStream_t st, int sm_count)
{
    int B = 0;
    int smem = sell_block<KP, NS>(B);
    if (MASK == 2) smem += p.mask_words * 4;
    const int64_t spb = B / (32 * NS);   // slices per block
    int64_t grid = (nslices + spb - 1) / spb;
    // no more blocks than fit at once: the warps loop over the slices
    const int occ = g_sell_per_sm[KP][NS][MASK];
    const int per_sm = occ > 0 ? occ : 1;
    if (grid > (int64_t)per_sm * sm_count) grid = (int64_t)per_sm * sm_count;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(B);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (carveout >= 0) {
        attr[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
        attr[0].val.sharedMemCarveout = (unsigned)carveout;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    if constexpr (NS == 1) return cudaLaunchKernelEx(&cfg, spmm_sell1_f32_kernel<KP, MASK>, p);
    else return cudaLaunchKernelEx(&cfg, spmm_sell_f32_kernel<KP, NS, MASK>, p);
}

template <int KP, int MASK>
static cudaError_t launch_f32_m(const SpmmParams<float>& p, int64_t nslices, SpmmConfig c,
                                cudaStream_t st, int sm_count)
{
    if constexpr (KP >= 16) {
        if (c.split == 4) return launch_f32_split<KP, 4, MASK>(p, nslices, c.carveout, st, sm_count);
        if (c.split == 2) return launch_f32_split<KP, 2, MASK>(p, nslices, c.carveout, st, sm_count);
    }
    return launch_f32_split<KP, 1, MASK>(p, nslices, c.carveout, st, sm_count);
}

template <int KP>
static cudaError_t launch_f32(const SpmmParams<float>& p, int64_t nslices, SpmmConfig c,
                              cudaStream_t st, int sm_count)
{
    if (c.mask == 2) {
        if (p.mask_words > kSellSmemMaskWords) return cudaErrorInvalidValue;
        return launch_f32_m<KP, 2>(p, nslices, c, st, sm_count);
    }
    return c.mask ? launch_f32_m<KP, 1>(p, nslices, c, st, sm_count)
                  : launch_f32_m<KP, 0>(p, nslices, c, st, sm_count);
}

template <typename T>
cudaError_t launch_spmm(const SellDev& S, const EllDev& F, int k, T* Y,
                        int64_t ldy, SpmmConfig cfg, cudaStream_t st, int sm_count)
{
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
    p.fmask = F.nzmask;
    p.mask_words = (int)((F.rows + 31) / 32);
    p.dld = F.dld;
    p.fld = F.ld;
    p.heavy = F.heavy;
    p.k = k;
    p.Y = Y;
    p.partials = static_cast<T*>(S.partials);
    p.frows = F.rows;
    p.yrows = S.rows;
    p.npart = S.npart;
    const int KP = F.ld;
    if constexpr (sizeof(T) == 4) {
        switch (KP) {
#define ESPNMF_KP(v) case v: return launch_f32<v>(p, S.nslices, cfg, st, sm_count);
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
static cudaError_t launch_freq(const FreqParams& p, int grid, bool global, cudaStream_t st)
{
    if (global) {
        spmm_freq_f32_kernel<KP, true><<<grid, kHThreads, kFreqRingBytes, st>>>(p);
    } else {
        // the table, a zero row and the rings
        const size_t smem = (size_t)(p.h + 1) * KP * 4 + kFreqRingBytes;
        spmm_freq_f32_kernel<KP, false><<<grid, kHThreads, smem, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_spmm_h(const SellDev& S, const EllDev& F, float* Y, int sm_count,
                          unsigned* status, long long wait_limit, cudaStream_t st, int tier)
{
    const bool global = tier == 2;
    const FreqTierDev& T = S.ft[global ? 1 : 0];
    if (S.h <= 0 || T.nrows == 0 || (global && S.h <= S.h1)) return cudaSuccess;
    if (F.htab == nullptr || F.h != S.h) return cudaErrorInvalidValue;
    FreqParams p;
    p.ent = T.ent;
    p.rows = T.rows;
    p.chunk = T.chunk;
    p.nchunks = T.nchunks;
    p.counter = T.counter;
    p.htab = static_cast<const float*>(F.htab);
    p.h = global ? S.h : S.h1;
    p.Y = Y;
    p.status = status;
    p.wait_limit = wait_limit < (1ll << 20) ? wait_limit : (1ll << 20);
    const int grid = sm_count;
    if (!global && (size_t)S.h1 * F.ld * 4 > kHTableBytes) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(p.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    switch (F.ld) {
#define ESPNMF_KP(v) case v: return launch_freq<v>(p, grid, global, st);
        ESPNMF_KP(4) ESPNMF_KP(8) ESPNMF_KP(12) ESPNMF_KP(16) ESPNMF_KP(20) ESPNMF_KP(24)
        ESPNMF_KP(28) ESPNMF_KP(32) ESPNMF_KP(36) ESPNMF_KP(40) ESPNMF_KP(44) ESPNMF_KP(48)
        ESPNMF_KP(52) ESPNMF_KP(56) ESPNMF_KP(60) ESPNMF_KP(64) ESPNMF_KP(80) ESPNMF_KP(96)
        ESPNMF_KP(112) ESPNMF_KP(128)
#undef ESPNMF_KP
    default: return cudaErrorInvalidValue;
    }
}

template <typename K>
static cudaError_t setup_sell_kernel(K kern, int B, int smem, int& per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, (size_t)smem);
}

template <int KP, int NS, int MASK>
static cudaError_t setup_sell_one()
{
    int B = 0;
    const int smem = sell_block<KP, NS>(B);
    int per_sm = 0;
    cudaError_t e;
    if constexpr (NS == 1) e = setup_sell_kernel(spmm_sell1_f32_kernel<KP, MASK>, B, smem, per_sm);
    else e = setup_sell_kernel(spmm_sell_f32_kernel<KP, NS, MASK>, B, smem, per_sm);
    g_sell_per_sm[KP][NS][MASK] = per_sm;
    return e;
}

template <int KP, int NS>
static cudaError_t setup_sell_occupancy()
{
    cudaError_t e = setup_sell_one<KP, NS, 0>();
    if (e == cudaSuccess) e = setup_sell_one<KP, NS, 1>();
    if (e == cudaSuccess) e = setup_sell_one<KP, NS, 2>();
    return e;
}

template <int KP>
static cudaError_t setup_f32()
{
    // the largest table (kHTableBytes and a row), its zero row and the rings
    cudaError_t e = cudaFuncSetAttribute(spmm_freq_f32_kernel<KP, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kHTableBytes + 2 * KP * 4 + kFreqRingBytes));
    if constexpr (KP >= 16) {
        if (e == cudaSuccess) e = setup_sell_occupancy<KP, 2>();
        if (e == cudaSuccess) e = setup_sell_occupancy<KP, 4>();
    }
    if (e == cudaSuccess) e = setup_sell_occupancy<KP, 1>();
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

ESPNMF_CHECK_READER(check_flags_spmm)

template cudaError_t launch_spmm<float>(const SellDev&, const EllDev&, int, float*, int64_t, SpmmConfig, cudaStream_t, int);
template cudaError_t launch_spmm<double>(const SellDev&, const EllDev&, int, double*, int64_t, SpmmConfig, cudaStream_t, int);
template cudaError_t launch_spmm_combine<float>(const SellDev&, int, float*, int64_t, cudaStream_t);
template cudaError_t launch_spmm_combine<double>(const SellDev&, int, double*, int64_t, cudaStream_t);

}  // namespace espnmf
