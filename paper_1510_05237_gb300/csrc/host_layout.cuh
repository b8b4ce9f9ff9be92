// host_layout.cuh -- the host-side layouts of A for the sparse products
// of Alg. 2 steps 1 and 3, built by espnmf_init on host threads:
//
//   * transpose_csr: the CSC of A (= CSR of A^T), a counting sort;
//   * build_sell:    the SELL-32x4 layout of a CSR matrix;
//   * choose_frequent / split_frequent / balance_frequent: the FP32 form's
//     frequent part (the entries whose gathered factor row is one of the
//     most referenced ones), in two tiers, and the rest for build_sell;
//   * build_layouts_f32: both orientations of the FP32 form;
//   * pack_factor:   a row-packed factor in an export layout
//     (espnmf_get_factor).
//
// Host code only (no CUDA calls); the vector types come from the CUDA
// headers.  The device side of these layouts is described with SellDev and
// FreqTierDev in common.cuh.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "../../include/espnmf.h"
#include "common.cuh"

namespace espnmf {
namespace layout {

// Host threads for one parallel pass: all hardware threads (at most 32),
// or half of them inside one of the two layout builds that run at once.
inline thread_local int t_share = 1;
inline int host_threads()
{
    const unsigned hw = std::thread::hardware_concurrency();
    const int all = (int)std::min<unsigned>(32u, hw ? hw : 1u);
    return std::max(1, all / t_share);
}

// fn(lo, hi) over [0, total) cut into contiguous chunks run on the host
// threads (one for small totals).
template <typename F>
void parallel_chunks(int64_t total, F&& fn)
{
    int T = host_threads();
    if (total < (1 << 16)) T = 1;
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t)
        th.emplace_back([&, t] { fn(total * t / T, total * (t + 1) / T); });
    fn(0, total / T);
    for (auto& x : th) x.join();
}

// fn(lo, hi) over [0, total) cut into contiguous chunks of about equal
// weight, where prefix[i] is the weight of items [0, i) (row pointers, slice
// pointers), on up to eight host threads.
template <typename F>
void parallel_weighted(int64_t total, const int64_t* prefix, F&& fn)
{
    int T = host_threads();
    const int64_t W = prefix[total] - prefix[0];
    if (W < (1 << 16) || total < 2) T = 1;
    std::vector<int64_t> cut(T + 1, total);
    cut[0] = 0;
    for (int t = 1; t < T; ++t)
        cut[t] = std::lower_bound(prefix, prefix + total + 1, prefix[0] + W * t / T) - prefix;
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t)
        if (cut[t] < cut[t + 1]) th.emplace_back([&, t] { fn(cut[t], cut[t + 1]); });
    if (cut[0] < cut[1]) fn(cut[0], cut[1]);
    for (auto& x : th) x.join();
}

// Host vectors whose resize leaves the new elements uninitialised (every
// element is written by the parallel passes that follow), so that building
// a layout does not pay a serial zero-fill of each buffer first.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <typename U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <typename U>
    void construct(U* p) noexcept
    {
        ::new (static_cast<void*>(p)) U;
    }
    template <typename U, typename... Args>
    void construct(U* p, Args&&... args)
    {
        ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
    }
};
template <typename T>
using hvec = std::vector<T, NoInitAlloc<T>>;

// CSC of an n x m CSR matrix (= CSR of its transpose, values converted to
// VO), rows ascending inside each column: a counting sort by column over
// row ranges of about equal nnz, one per host thread.  Thread t's entries of
// column j are placed after those of threads < t, so every column lists its
// rows in ascending order, exactly as one serial pass would.
template <typename VI, typename VO>
void transpose_csr(int64_t n, int64_t m, const int64_t* rp, const int32_t* ci, const VI* vv,
                   std::vector<int64_t>& cp, hvec<int32_t>& ri, hvec<VO>& cv)
{
    const int64_t nnz = rp[n];
    int T = host_threads();
    if (nnz < (1 << 18)) T = 1;
    std::vector<int64_t> r0(T + 1, n);
    r0[0] = 0;
    for (int t = 1; t < T; ++t)
        r0[t] = std::lower_bound(rp, rp + n + 1, nnz * t / T) - rp;
    std::vector<std::vector<int64_t>> off(T);
    auto on_threads = [&](auto&& fn) {
        std::vector<std::thread> th;
        for (int t = 1; t < T; ++t) th.emplace_back([&, t] { fn(t); });
        fn(0);
        for (auto& x : th) x.join();
    };
    on_threads([&](int t) {
        off[t].assign(m, 0);
        int64_t* c = off[t].data();
        for (int64_t p = rp[r0[t]]; p < rp[r0[t + 1]]; ++p) c[ci[p]]++;
    });
    cp.assign(m + 1, 0);
    parallel_chunks(m, [&](int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; ++j) {
            int64_t s = 0;
            for (int t = 0; t < T; ++t) s += off[t][j];
            cp[j + 1] = s;
        }
    });
    for (int64_t j = 0; j < m; ++j) cp[j + 1] += cp[j];
    parallel_chunks(m, [&](int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; ++j) {
            int64_t base = cp[j];
            for (int t = 0; t < T; ++t) {
                const int64_t c = off[t][j];
                off[t][j] = base;
                base += c;
            }
        }
    });
    ri.resize(nnz);
    cv.resize(nnz);
    on_threads([&](int t) {
        int64_t* o = off[t].data();
        for (int64_t r = r0[t]; r < r0[t + 1]; ++r)
            for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
                const int64_t q = o[ci[p]]++;
                ri[q] = (int32_t)r;
                cv[q] = (VO)vv[p];
            }
    });
}

// --- host-side layout of A ------------------------------------------------------

template <typename T>
struct SellHost {
    int64_t rows = 0, nseg = 0, nslices = 0, total = 0, nnz = 0, npart = 0;
    std::vector<int64_t> slice_ptr;
    std::vector<int32_t> slice_len, seg_row, seg_part, seg_grp, split_row, split_first,
        split_count;
    hvec<int32_t> idx;
    hvec<T> val;
};

// Lays out the rows of a CSR matrix for spmm_sell.  Every row becomes a
// group of 1..32 segments of at most kSegTarget entries (split evenly),
// placed in adjacent lanes of one 32-lane slice, so the lanes' partial sums
// are combined inside the warp.  A row with more than 32*kSegTarget entries
// is cut into chunks of up to 32 segments; each chunk writes a partial row
// that spmm_combine adds in chunk order.  Groups are sorted by segment
// length (longest first) and packed greedily, so the lanes of a slice walk
// segments of about the same length.  Entry p of lane l of slice s is
// stored at slice_ptr[s] + (p / 4) * 128 + 4 l + p % 4 (SELL-32 with groups
// of four), so each lane reads four entries with one 16-byte load and a
// warp reads 512 consecutive bytes.
template <typename T, typename V>
void build_sell(int64_t rows, const int64_t* ptr, const int32_t* ind, const V* vals,
                SellHost<T>& S)
{
    struct Grp {
        int32_t row, part, nseg, seglen;
        int64_t start, len;
    };
    std::vector<Grp> grps;
    grps.reserve((size_t)rows + 16);
    int64_t npart = 0;
    auto ceil_div = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
    for (int64_t r = 0; r < rows; ++r) {
        const int64_t len = ptr[r + 1] - ptr[r];
        const int64_t nseg = std::max<int64_t>(1, ceil_div(len, kSegTarget));
        if (nseg <= 32) {
            grps.push_back({(int32_t)r, -1, (int32_t)nseg, (int32_t)ceil_div(len, nseg), ptr[r], len});
        } else {
            const int64_t nch = ceil_div(nseg, 32);
            S.split_row.push_back((int32_t)r);
            S.split_first.push_back((int32_t)npart);
            S.split_count.push_back((int32_t)nch);
            for (int64_t c = 0; c < nch; ++c) {
                const int64_t s0 = len * c / nch, s1 = len * (c + 1) / nch, cl = s1 - s0;
                const int64_t ns = std::min<int64_t>(32, std::max<int64_t>(1, ceil_div(cl, kSegTarget)));
                grps.push_back({(int32_t)r, (int32_t)npart++, (int32_t)ns, (int32_t)ceil_div(cl, ns),
                                ptr[r] + s0, cl});
            }
        }
    }
    // counting sort by segment length, longest first, stable
    std::vector<int64_t> bucket(kSegTarget + 2, 0);
    for (auto& g : grps) bucket[kSegTarget - g.seglen + 1]++;
    for (int i = 1; i < kSegTarget + 2; ++i) bucket[i] += bucket[i - 1];
    std::vector<Grp> sorted(grps.size());
    for (auto& g : grps) sorted[bucket[kSegTarget - g.seglen]++] = g;
    // pack groups into slices
    struct Lane {
        int32_t row, part, grp, len;
        int64_t start;
    };
    std::vector<Lane> lanes;
    lanes.reserve(sorted.size() * 2 + 32);
    int used = 0;
    auto pad_to_slice = [&]() {
        while (used % 32 != 0) {
            lanes.push_back({-1, -1, ((used % 32) << 8) | ((used % 32) + 1), 0, 0});
            ++used;
        }
    };
    for (auto& g : sorted) {
        if ((used % 32) + g.nseg > 32) pad_to_slice();
        const int head = used % 32;
        for (int q = 0; q < g.nseg; ++q) {
            const int64_t a0 = g.len * q / g.nseg, a1 = g.len * (q + 1) / g.nseg;
            lanes.push_back({g.row, g.part, (head << 8) | (head + g.nseg), (int32_t)(a1 - a0),
                             g.start + a0});
            ++used;
        }
    }
    pad_to_slice();
    S.rows = rows;
    S.nnz = ptr[rows];
    S.npart = npart;
    S.nseg = (int64_t)lanes.size();
    S.nslices = S.nseg / 32;
    S.slice_ptr.assign(S.nslices + 1, 0);
    S.slice_len.assign(S.nslices, 0);
    // a slice's length is its longest segment rounded up to 4: each lane's
    // entries are stored in groups of four, so a 16-byte load brings four
    for (int64_t s = 0; s < S.nslices; ++s) {
        int mx = 0;
        for (int l = 0; l < 32; ++l) mx = std::max(mx, lanes[s * 32 + l].len);
        mx = (mx + 3) / 4 * 4;
        S.slice_len[s] = mx;
        S.slice_ptr[s + 1] = S.slice_ptr[s] + (int64_t)mx * 32;
    }
    S.total = S.slice_ptr[S.nslices];
    S.idx.resize(S.total);
    S.val.resize(S.total);
    S.seg_row.resize(S.nseg);
    S.seg_part.resize(S.nseg);
    S.seg_grp.resize(S.nseg);
    // slices in parallel (chunks of about equal storage): padding first,
    // then each lane's entries
    parallel_weighted(S.nslices, S.slice_ptr.data(), [&](int64_t s0, int64_t s1) {
        for (int64_t s = s0; s < s1; ++s) {
            std::fill(S.idx.begin() + S.slice_ptr[s], S.idx.begin() + S.slice_ptr[s + 1], -1);
            std::fill(S.val.begin() + S.slice_ptr[s], S.val.begin() + S.slice_ptr[s + 1], T(0));
            for (int64_t g = s * 32; g < s * 32 + 32; ++g) {
                const Lane& ln = lanes[g];
                S.seg_row[g] = ln.row;
                S.seg_part[g] = ln.part;
                S.seg_grp[g] = ln.grp;
                const int64_t o = S.slice_ptr[s] + (g % 32) * 4;
                for (int p = 0; p < ln.len; ++p) {
                    const int64_t at = o + (int64_t)(p / 4) * 128 + p % 4;
                    S.idx[at] = ind[ln.start + p];
                    S.val[at] = (T)vals[ln.start + p];
                }
            }
        }
    });
}

// The frequent part of an FP32 product.  The gathered rows that the most
// entries reference (weight = entries per gathered row) are candidates when
// they are referenced at least 4x as often as the average row (and at least
// 16 times), in decreasing weight (ties: lower index first).  The first
// kHTableBytes / (ld * 4) of them form the table staged in shared memory
// (tier 1).  Column enforcement keeps t rows per factor column, so at most
// t gathered rows can be nonzero in every column: with t_rows = t (0 in the
// other modes) the table takes up to t candidates, those beyond tier 1
// read from global memory (tier 2, kept only if it holds at least
// kMinTier2Rows rows; at most kH2TableBytes and 2^16 - 1 rows in all).  The
// part is kept only if its entries are at least a tenth of all.  Returns h
// (0: none), sets h1 (rows in tier 1) and fills slot_of.
inline int choose_frequent(const std::vector<int64_t>& weight, int64_t nnz, int ld, int64_t t_rows,
                    std::vector<int32_t>& slot_of, int& h1)
{
    const int64_t ng = (int64_t)weight.size();
    slot_of.assign(ng, -1);
    h1 = 0;
    if (ng == 0 || nnz == 0) return 0;
    const int64_t cap1 = std::min<int64_t>((int64_t)(kHTableBytes / ((size_t)ld * 4)), 65535);
    const int64_t cap_all = std::min<int64_t>((int64_t)(kH2TableBytes / ((size_t)ld * 4)), 65535);
    const double floor_w = std::max(16.0, 4.0 * (double)nnz / (double)ng);
    std::vector<int32_t> order;
    for (int64_t g = 0; g < ng; ++g)
        if ((double)weight[g] >= floor_w) order.push_back((int32_t)g);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return weight[a] > weight[b]; });
    int64_t cap = cap1;
    const int64_t want = std::min<int64_t>({(int64_t)order.size(), t_rows, cap_all});
    if (want - cap1 >= kMinTier2Rows) cap = want;
    if ((int64_t)order.size() > cap) order.resize(cap);
    int64_t covered = 0;
    for (int32_t g : order) covered += weight[g];
    if (order.empty() || covered * 10 < nnz) return 0;
    for (size_t q = 0; q < order.size(); ++q) slot_of[order[q]] = (int32_t)q;
    h1 = (int)std::min<int64_t>((int64_t)order.size(), cap1);
    return (int)order.size();
}

// Splits a CSR matrix into the entries of frequent gathered rows, per tier
// and output row as (byte offset of the gathered row in its table, value)
// padded with entries on the zero row to a multiple of freq_pad(ld), and
// the rest (a CSR matrix for build_sell, its values rounded to FP32 as the
// layout stores them).  False (nothing built) if a tier's entries exceed
// what its 32-bit row ends can address.
struct FreqTierHost {
    std::vector<int64_t> ptr;      // [rows + 1] stored entries before each output row
    hvec<uint2> ent;
    std::vector<int2> rows;        // (output row, end / 4) of the rows with entries
    std::vector<int32_t> chunk;
    int64_t nnz = 0;
};
struct FreqHost {
    int h = 0, h1 = 0;
    std::vector<int32_t> slot_of;
    FreqTierHost t[2];             // slots < h1 (staged); slots h1 .. h - 1
};

template <typename V>
bool split_frequent(int64_t rows, const int64_t* ptr, const int32_t* ind, const V* vals,
                    int ld, FreqHost& F, std::vector<int64_t>& lptr, hvec<int32_t>& lind,
                    hvec<float>& lval)
{
    const int64_t pad = freq_pad(ld);
    const uint32_t row_bytes = (uint32_t)ld * 4u;
    const int h1 = F.h1;
    // the zero row: after the staged rows (tier 1), the factor table's row h
    // (tier 2)
    const uint32_t zero_off[2] = {(uint32_t)h1 * row_bytes, (uint32_t)F.h * row_bytes};
    std::vector<int64_t> cnt[2];
    for (int u = 0; u < 2; ++u) {
        F.t[u].ptr.assign(rows + 1, 0);
        cnt[u].assign(rows, 0);
    }
    lptr.assign(rows + 1, 0);
    parallel_weighted(rows, ptr, [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; ++r) {
            int64_t n1 = 0, n2 = 0;
            for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) {
                const int32_t sl = F.slot_of[ind[q]];
                n1 += sl >= 0 && sl < h1;
                n2 += sl >= h1;
            }
            cnt[0][r] = n1;
            cnt[1][r] = n2;
            F.t[0].ptr[r + 1] = (n1 + pad - 1) / pad * pad;
            F.t[1].ptr[r + 1] = (n2 + pad - 1) / pad * pad;
            lptr[r + 1] = ptr[r + 1] - ptr[r] - n1 - n2;
        }
    });
    for (int64_t r = 0; r < rows; ++r) {
        for (int u = 0; u < 2; ++u) {
            F.t[u].ptr[r + 1] += F.t[u].ptr[r];
            F.t[u].nnz += cnt[u][r];
        }
        lptr[r + 1] += lptr[r];
    }
    for (int u = 0; u < 2; ++u)
        if (F.t[u].ptr[rows] / 4 > (int64_t)INT32_MAX) return false;
    for (int u = 0; u < 2; ++u) F.t[u].ent.resize(F.t[u].ptr[rows]);
    lind.resize(lptr[rows]);
    lval.resize(lptr[rows]);
    parallel_weighted(rows, ptr, [&](int64_t r0, int64_t r1) {
        for (int64_t r = r0; r < r1; ++r) {
            int64_t at[2] = {F.t[0].ptr[r], F.t[1].ptr[r]};
            int64_t b = lptr[r];
            for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) {
                const int32_t sl = F.slot_of[ind[q]];
                const float v = (float)vals[q];
                if (sl >= 0) {
                    const int u = sl < h1 ? 0 : 1;
                    uint32_t vb;
                    std::memcpy(&vb, &v, 4);
                    F.t[u].ent[at[u]++] = make_uint2((uint32_t)sl * row_bytes, vb);
                } else {
                    lind[b] = ind[q];
                    lval[b++] = v;
                }
            }
            for (int u = 0; u < 2; ++u)
                for (; at[u] < F.t[u].ptr[r + 1]; ++at[u])
                    F.t[u].ent[at[u]] = make_uint2(zero_off[u], 0u);
        }
    });
    for (int u = 0; u < 2; ++u) {
        FreqTierHost& T = F.t[u];
        for (int64_t r = 0; r < rows; ++r)
            if (T.ptr[r + 1] > T.ptr[r]) T.rows.push_back(make_int2((int)r, (int)(T.ptr[r + 1] / 4)));
    }
    return true;
}

// Chunks of a tier's rows for the warps of spmm_freq: contiguous ranges of
// about equal cost (entries, plus a fixed cost per row).
inline void balance_tier(int nchunks, FreqTierHost& T)
{
    const int64_t nr = (int64_t)T.rows.size();
    std::vector<int64_t> cost(nr + 1, 0);
    int64_t prev = 0;
    for (int64_t j = 0; j < nr; ++j) {
        const int64_t end = 4ll * T.rows[j].y;
        cost[j + 1] = cost[j] + (end - prev) + 8;
        prev = end;
    }
    T.chunk.assign(nchunks + 1, 0);
    int64_t j = 0;
    for (int c = 1; c < nchunks; ++c) {
        const double target = (double)cost[nr] * c / nchunks;
        while (j < nr && (double)cost[j] < target) ++j;
        T.chunk[c] = (int32_t)j;
    }
    T.chunk[nchunks] = (int32_t)nr;
}

inline void balance_frequent(int nchunks, FreqHost& F)
{
    balance_tier(nchunks, F.t[0]);
    if (F.h > F.h1) balance_tier(nchunks, F.t[1]);
}

// One orientation's FP32 layouts: the frequent part when its gathered rows
// are skewed enough (the frequent terms of a corpus), and the SELL part.
// optr: the other orientation's row pointers, whose row lengths are the
// entries that reference each gathered row; t_rows: the gathered factor's t
// per column in column mode (the most rows that can be nonzero in all of
// its columns), else 0.  vals in either precision: the layouts hold them
// rounded to FP32.
struct BuiltF32 {
    FreqHost F;
    SellHost<float> h;
};

template <typename V>
void build_f32(int64_t rows, const int64_t* ptr, const int32_t* ind, const V* vals,
               int64_t ngather, const int64_t* optr, int64_t t_rows, int ld, int nchunks,
               BuiltF32& B)
{
    std::vector<int64_t> w(ngather);
    for (int64_t g = 0; g < ngather; ++g) w[g] = optr[g + 1] - optr[g];
    B.F.h = choose_frequent(w, ptr[rows], ld, t_rows, B.F.slot_of, B.F.h1);
    std::vector<int64_t> lp;
    hvec<int32_t> li;
    hvec<float> lv;   // the rest's values, already rounded as the layout stores them
    if (B.F.h > 0 && !split_frequent(rows, ptr, ind, vals, ld, B.F, lp, li, lv))
        B.F = FreqHost{};
    if (B.F.h > 0) {
        balance_frequent(nchunks, B.F);
        build_sell(rows, lp.data(), li.data(), lv.data(), B.h);
    } else {
        build_sell(rows, ptr, ind, vals, B.h);
    }
}

// Both orientations on two host threads: rows of A (values va) gather rows
// of V (documents), rows of A^T (CSR cp, ri, vt) rows of U (terms).
template <typename VA, typename VT>
void build_layouts_f32(int64_t n, int64_t m, const int64_t* rp, const int32_t* ci, const VA* va,
                       const int64_t* cp, const int32_t* ri, const VT* vt, int ld, int nchunks,
                       int64_t t_u, int64_t t_v, BuiltF32& ba, BuiltF32& bat)
{
    std::thread th([&] {
        t_share = 2;
        build_f32(m, cp, ri, vt, n, rp, t_u, ld, nchunks, bat);
    });
    t_share = 2;
    build_f32(n, rp, ci, va, m, cp, t_v, ld, nchunks, ba);
    t_share = 1;
    th.join();
}


// A factor in row-packed form (row r: cnt[r] pairs (col, val) at
// [r * ld, r * ld + cnt[r]), columns distinct) written in an export layout
// with values of es bytes (8: FP64, 4: FP32, rounded from V):
//   DENSE_ROWMAJOR: vo = rows x k values, zeros included;
//   CSC: po[k + 1], io = rows ascending within each column;
//   CSR: po[rows + 1], io = columns ascending within each row.
// False for an unknown layout.
template <typename V>
bool pack_factor(int64_t rows, int k, int ld, const int32_t* cnt, const int32_t* col,
                 const V* val, espnmf_layout layout, size_t es, std::vector<unsigned char>& vo,
                 std::vector<int64_t>& po, std::vector<int32_t>& io)
{
    auto put = [&](size_t i, V x) {
        if (es == 8) {
            const double d = (double)x;
            std::memcpy(&vo[i * 8], &d, 8);
        } else {
            const float f = (float)x;
            std::memcpy(&vo[i * 4], &f, 4);
        }
    };
    int64_t nnz = 0;
    for (int64_t r = 0; r < rows; ++r) nnz += cnt[r];
    vo.clear();
    po.clear();
    io.clear();
    if (layout == ESPNMF_DENSE_ROWMAJOR) {
        vo.assign((size_t)rows * k * es, 0);
        for (int64_t r = 0; r < rows; ++r)
            for (int q = 0; q < cnt[r]; ++q)
                put((size_t)r * k + col[r * ld + q], val[r * ld + q]);
    } else if (layout == ESPNMF_CSR) {
        po.assign(rows + 1, 0);
        io.resize(nnz);
        vo.resize(nnz * es);
        int64_t o = 0;
        std::vector<std::pair<int32_t, V>> tmp;
        for (int64_t r = 0; r < rows; ++r) {
            tmp.clear();
            for (int q = 0; q < cnt[r]; ++q) tmp.push_back({col[r * ld + q], val[r * ld + q]});
            std::sort(tmp.begin(), tmp.end());
            for (auto& pr : tmp) {
                io[o] = pr.first;
                put(o, pr.second);
                ++o;
            }
            po[r + 1] = o;
        }
    } else if (layout == ESPNMF_CSC) {
        po.assign(k + 1, 0);
        for (int64_t r = 0; r < rows; ++r)
            for (int q = 0; q < cnt[r]; ++q) po[col[r * ld + q] + 1]++;
        for (int c = 0; c < k; ++c) po[c + 1] += po[c];
        std::vector<int64_t> nx(po.begin(), po.end() - 1);
        io.resize(nnz);
        vo.resize(nnz * es);
        for (int64_t r = 0; r < rows; ++r)   // rows ascending -> sorted columns
            for (int q = 0; q < cnt[r]; ++q) {
                const int c = col[r * ld + q];
                const int64_t o = nx[c]++;
                io[o] = (int32_t)r;
                put(o, val[r * ld + q]);
            }
    } else {
        return false;
    }
    return true;
}

}  // namespace layout
}  // namespace espnmf
