// Host-side check of the layouts of A that espnmf_init builds
// (paper_1510_05237_gb300/csrc/host_layout.cuh), with no GPU:
//
//   1. transpose_csr against a serial transpose (FP32 and FP64 values);
//   2. the FP32 form's layouts of both orientations built from FP32 values
//      and from the same values widened to FP64: bitwise equal;
//   3. every entry of A, and nothing else, recovered from each orientation's
//      SELL part and the two tiers of its frequent part, each with its row,
//      column and FP32 value; the tiers' padding, row list and work chunks
//      well formed;
//   4. pack_factor (the export of a row-packed factor) against a dense
//      reference in all three layouts, FP32 and FP64 values and outputs.
//
// Usage: host_layout_check <prefix> <n> <m> <ld> <t_u> <t_v>
// reads <prefix>_rp.bin (int64[n+1]), <prefix>_ci.bin (int32[nnz]) and
// <prefix>_vf.bin (float[nnz]); prints one summary line; exit status 0 when
// every check holds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "host_layout.cuh"

// The padding multiple of a tier's rows, as the frequent-part kernel steps
// through them: lanes per entry = the power of two >= ld / 4 (at least two),
// 2 * 32 / lanes entries per warp step, at least four.
int espnmf::freq_pad(int ld)
{
    const int q = ld / 4;
    const int lanes = q <= 2 ? 2 : q <= 4 ? 4 : q <= 8 ? 8 : q <= 16 ? 16 : 32;
    const int step = 2 * (32 / lanes);
    return step > 4 ? step : 4;
}

using namespace espnmf;
using namespace espnmf::layout;

namespace {

int g_fail = 0;
void fail(const char* what)
{
    if (g_fail++ < 10) std::printf("FAIL: %s\n", what);
}

template <class T>
std::vector<T> read_bin(const char* path)
{
    std::vector<T> v;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return v;
    std::fseek(fp, 0, SEEK_END);
    const long sz = std::ftell(fp);
    std::fseek(fp, 0, SEEK_SET);
    v.resize((size_t)sz / sizeof(T));
    if (std::fread(v.data(), 1, (size_t)sz, fp) != (size_t)sz) v.clear();
    std::fclose(fp);
    return v;
}

template <class A, class B>
bool same(const A& a, const B& b)
{
    return a.size() == b.size() &&
           (a.empty() || std::memcmp(a.data(), b.data(), a.size() * sizeof(a[0])) == 0);
}

bool same_sell(const SellHost<float>& a, const SellHost<float>& b)
{
    return a.rows == b.rows && a.nseg == b.nseg && a.nslices == b.nslices && a.total == b.total &&
           a.nnz == b.nnz && a.npart == b.npart && same(a.slice_ptr, b.slice_ptr) &&
           same(a.slice_len, b.slice_len) && same(a.seg_row, b.seg_row) &&
           same(a.seg_part, b.seg_part) && same(a.seg_grp, b.seg_grp) &&
           same(a.split_row, b.split_row) && same(a.split_first, b.split_first) &&
           same(a.split_count, b.split_count) && same(a.idx, b.idx) && same(a.val, b.val);
}

bool same_freq(const FreqHost& a, const FreqHost& b)
{
    bool ok = a.h == b.h && a.h1 == b.h1 && same(a.slot_of, b.slot_of);
    for (int u = 0; u < 2; ++u)
        ok = ok && same(a.t[u].ptr, b.t[u].ptr) && same(a.t[u].ent, b.t[u].ent) &&
             same(a.t[u].rows, b.t[u].rows) && same(a.t[u].chunk, b.t[u].chunk) &&
             a.t[u].nnz == b.t[u].nnz;
    return ok;
}

// CSC by one serial pass: column by column, rows ascending
template <class V>
void serial_transpose(int64_t n, int64_t m, const std::vector<int64_t>& rp,
                      const std::vector<int32_t>& ci, const V* vv, std::vector<int64_t>& cp,
                      std::vector<int32_t>& ri, std::vector<V>& cv)
{
    cp.assign(m + 1, 0);
    for (int64_t p = 0; p < rp[n]; ++p) cp[ci[p] + 1]++;
    for (int64_t j = 0; j < m; ++j) cp[j + 1] += cp[j];
    std::vector<int64_t> at(cp.begin(), cp.end() - 1);
    ri.resize(rp[n]);
    cv.resize(rp[n]);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
            ri[at[ci[p]]] = (int32_t)r;
            cv[at[ci[p]]++] = vv[p];
        }
}

struct Entry {
    int64_t row;
    int32_t col;
    float val;
    bool operator<(const Entry& o) const { return std::tie(row, col) < std::tie(o.row, o.col); }
};

// Every (row, column, value) held by one orientation's FP32 layouts, and
// the structural checks of its frequent part.
std::vector<Entry> recover(const BuiltF32& B, int ld, int64_t ngather)
{
    std::vector<Entry> out;
    const SellHost<float>& S = B.h;
    for (int64_t s = 0; s < S.nslices; ++s)
        for (int l = 0; l < 32; ++l) {
            const int32_t row = S.seg_row[s * 32 + l];
            for (int p = 0; p < S.slice_len[s]; ++p) {
                const int64_t at = S.slice_ptr[s] + (int64_t)(p / 4) * 128 + 4 * l + p % 4;
                if (S.idx[at] < 0) continue;
                if (row < 0) fail("entry in a padding lane");
                out.push_back({row, S.idx[at], S.val[at]});
            }
        }
    const FreqHost& F = B.F;
    if (F.h == 0) return out;
    if (F.h1 < 1 || F.h1 > F.h) fail("tier sizes");
    std::vector<int64_t> gathered(F.h, -1);
    for (int64_t g = 0; g < ngather; ++g) {
        const int32_t sl = F.slot_of[g];
        if (sl < -1 || sl >= F.h) fail("slot out of range");
        else if (sl >= 0) {
            if (gathered[sl] >= 0) fail("slot given twice");
            gathered[sl] = g;
        }
    }
    for (int32_t sl = 0; sl < F.h; ++sl)
        if (gathered[sl] < 0) fail("slot without a gathered row");
    const uint32_t row_bytes = (uint32_t)ld * 4u;
    const int pad = freq_pad(ld);
    for (int u = 0; u < 2; ++u) {
        const FreqTierHost& T = F.t[u];
        const uint32_t zero_off = (uint32_t)(u == 0 ? F.h1 : F.h) * row_bytes;
        const int32_t lo = u == 0 ? 0 : F.h1, hi = u == 0 ? F.h1 : F.h;
        int64_t prev = 0, nnz = 0, last_row = -1;
        for (const int2& r : T.rows) {
            const int64_t end = 4ll * r.y;
            if (r.x <= last_row) fail("tier rows not ascending");
            if (end <= prev || (end - prev) % pad != 0) fail("tier row not padded to the step");
            last_row = r.x;
            int64_t real = 0;
            for (int64_t e = prev; e < end; ++e) {
                const uint2 en = T.ent[e];
                if (en.x == zero_off) {
                    if (en.y != 0u) fail("padding entry with a value");
                    continue;
                }
                if (en.x % row_bytes != 0) fail("table offset not on a row");
                const int32_t sl = (int32_t)(en.x / row_bytes);
                if (sl < lo || sl >= hi) {
                    fail("slot outside its tier");
                    continue;
                }
                float v;
                std::memcpy(&v, &en.y, 4);
                out.push_back({r.x, (int32_t)gathered[sl], v});
                ++real;
            }
            if (real == 0 || end - prev - real >= pad) fail("tier row padding");
            nnz += real;
            prev = end;
        }
        if ((int64_t)T.ent.size() != prev) fail("tier entries beyond the last row");
        if (nnz != T.nnz) fail("tier entry count");
        if (!T.rows.empty()) {
            if (T.chunk.empty() || T.chunk.front() != 0 || T.chunk.back() != (int32_t)T.rows.size())
                fail("tier chunks do not cover the rows");
            for (size_t c = 1; c < T.chunk.size(); ++c)
                if (T.chunk[c] < T.chunk[c - 1]) fail("tier chunks not ascending");
        }
    }
    return out;
}

// (row, column, FP32 value) of a CSR matrix, in row-major order
std::vector<Entry> entries_of(int64_t rows, const int64_t* ptr, const int32_t* ind,
                              const float* val)
{
    std::vector<Entry> out;
    out.reserve(ptr[rows]);
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t p = ptr[r]; p < ptr[r + 1]; ++p) out.push_back({r, ind[p], val[p]});
    return out;
}

bool same_entries(std::vector<Entry> a, std::vector<Entry> b)
{
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a.size() != b.size()) return false;
    for (size_t q = 0; q < a.size(); ++q)
        if (a[q].row != b[q].row || a[q].col != b[q].col ||
            std::memcmp(&a[q].val, &b[q].val, 4) != 0)
            return false;
    return true;
}

// A random row-packed factor (rows x k, ld >= k, distinct columns per row,
// values > 0) exported by pack_factor and compared with a dense reference.
template <class V>
void check_pack(int64_t rows, int k, int ld, unsigned seed)
{
    uint64_t st = seed * 2654435761ull + 1;
    auto next = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return st;
    };
    std::vector<int32_t> cnt(rows), col((size_t)rows * ld, -7);
    std::vector<V> val((size_t)rows * ld, (V)-3);
    std::vector<double> dense((size_t)rows * k, 0.0);
    for (int64_t r = 0; r < rows; ++r) {
        std::vector<int32_t> perm(k);
        for (int c = 0; c < k; ++c) perm[c] = c;
        for (int c = k - 1; c > 0; --c) std::swap(perm[c], perm[next() % (uint64_t)(c + 1)]);
        cnt[r] = (int32_t)(next() % (uint64_t)(k + 1));
        for (int q = 0; q < cnt[r]; ++q) {
            const V x = (V)((double)(next() % 1000000 + 1) / 7.0);
            col[r * ld + q] = perm[q];
            val[r * ld + q] = x;
            dense[(size_t)r * k + perm[q]] = (double)x;
        }
    }
    for (size_t es : {size_t(4), size_t(8)}) {
        auto as = [&](double x, unsigned char* out) {
            if (es == 8) std::memcpy(out, &x, 8);
            else {
                const float f = (float)x;
                std::memcpy(out, &f, 4);
            }
        };
        std::vector<unsigned char> vo;
        std::vector<int64_t> po;
        std::vector<int32_t> io;
        // dense
        pack_factor(rows, k, ld, cnt.data(), col.data(), val.data(), ESPNMF_DENSE_ROWMAJOR, es,
                    vo, po, io);
        std::vector<unsigned char> ref(dense.size() * es);
        for (size_t i = 0; i < dense.size(); ++i) as(dense[i], &ref[i * es]);
        if (vo != ref || !po.empty() || !io.empty()) fail("pack_factor dense");
        // CSR: columns ascending per row
        std::vector<int64_t> rp{0};
        std::vector<int32_t> ri;
        std::vector<unsigned char> rv;
        for (int64_t r = 0; r < rows; ++r) {
            for (int c = 0; c < k; ++c)
                if (dense[(size_t)r * k + c] != 0.0) {
                    ri.push_back(c);
                    rv.resize(rv.size() + es);
                    as(dense[(size_t)r * k + c], &rv[rv.size() - es]);
                }
            rp.push_back((int64_t)ri.size());
        }
        pack_factor(rows, k, ld, cnt.data(), col.data(), val.data(), ESPNMF_CSR, es, vo, po, io);
        if (po != rp || io != ri || vo != rv) fail("pack_factor CSR");
        // CSC: rows ascending per column
        rp.assign(1, 0);
        ri.clear();
        rv.clear();
        for (int c = 0; c < k; ++c) {
            for (int64_t r = 0; r < rows; ++r)
                if (dense[(size_t)r * k + c] != 0.0) {
                    ri.push_back((int32_t)r);
                    rv.resize(rv.size() + es);
                    as(dense[(size_t)r * k + c], &rv[rv.size() - es]);
                }
            rp.push_back((int64_t)ri.size());
        }
        pack_factor(rows, k, ld, cnt.data(), col.data(), val.data(), ESPNMF_CSC, es, vo, po, io);
        if (po != rp || io != ri || vo != rv) fail("pack_factor CSC");
    }
    std::vector<unsigned char> vo;
    std::vector<int64_t> po;
    std::vector<int32_t> io;
    if (pack_factor(rows, k, ld, cnt.data(), col.data(), val.data(), (espnmf_layout)7, 4, vo, po,
                    io))
        fail("pack_factor accepted an unknown layout");
}

}  // namespace

int main(int argc, char** argv)
{
    if (argc != 7) {
        std::printf("usage: %s prefix n m ld t_u t_v\n", argv[0]);
        return 2;
    }
    const std::string pre = argv[1];
    const int64_t n = std::atoll(argv[2]), m = std::atoll(argv[3]);
    const int ld = std::atoi(argv[4]);
    const int64_t t_u = std::atoll(argv[5]), t_v = std::atoll(argv[6]);
    const auto rp = read_bin<int64_t>((pre + "_rp.bin").c_str());
    const auto ci = read_bin<int32_t>((pre + "_ci.bin").c_str());
    const auto vf = read_bin<float>((pre + "_vf.bin").c_str());
    if ((int64_t)rp.size() != n + 1 || (int64_t)ci.size() != rp[n] || vf.size() != ci.size()) {
        std::printf("FAIL: input files\n");
        return 2;
    }
    const int64_t nnz = rp[n];
    std::vector<double> vv(vf.begin(), vf.end());

    // 4. factor export (independent of A)
    check_pack<float>(1000, 13, 16, 1);
    check_pack<double>(1000, 13, 16, 2);
    check_pack<float>(300, 50, 52, 3);
    check_pack<double>(64, 1, 4, 4);
    check_pack<float>(0, 5, 8, 5);

    // 1. transposes
    std::vector<int64_t> cp0;
    std::vector<int32_t> ri0;
    std::vector<float> cv0;
    std::vector<double> cv0d;
    serial_transpose(n, m, rp, ci, vf.data(), cp0, ri0, cv0);
    serial_transpose(n, m, rp, ci, vv.data(), cp0, ri0, cv0d);
    std::vector<int64_t> cp;
    hvec<int32_t> ri;
    hvec<float> cv;
    transpose_csr(n, m, rp.data(), ci.data(), vf.data(), cp, ri, cv);
    if (!same(cp, cp0) || !same(ri, ri0) || !same(cv, cv0)) fail("transpose (FP32 values)");
    std::vector<int64_t> cpd;
    hvec<int32_t> rid;
    hvec<float> cvd;
    transpose_csr(n, m, rp.data(), ci.data(), vv.data(), cpd, rid, cvd);
    if (!same(cpd, cp0) || !same(rid, ri0) || !same(cvd, cv0)) fail("transpose (FP64 values)");
    hvec<double> cv64;
    transpose_csr(n, m, rp.data(), ci.data(), vv.data(), cpd, rid, cv64);
    if (!same(cv64, cv0d)) fail("transpose (FP64 form)");

    // 2. both orientations from FP32 and from FP64 values
    const int nchunks = 4 * 152 * 32;
    BuiltF32 a32, at32, a64, at64;
    build_layouts_f32(n, m, rp.data(), ci.data(), vf.data(), cp.data(), ri.data(), cv.data(), ld,
                      nchunks, t_u, t_v, a32, at32);
    build_layouts_f32(n, m, rp.data(), ci.data(), vv.data(), cp.data(), ri.data(), cv64.data(), ld,
                      nchunks, t_u, t_v, a64, at64);
    if (!same_sell(a32.h, a64.h) || !same_freq(a32.F, a64.F)) fail("A: FP32 vs FP64 values");
    if (!same_sell(at32.h, at64.h) || !same_freq(at32.F, at64.F)) fail("A^T: FP32 vs FP64 values");
    // FP64 input in the FP32 form: A's values in FP64, A^T's transposed to FP32
    BuiltF32 amix, atmix;
    build_layouts_f32(n, m, rp.data(), ci.data(), vv.data(), cpd.data(), rid.data(), cvd.data(),
                      ld, nchunks, t_u, t_v, amix, atmix);
    if (!same_sell(a32.h, amix.h) || !same_freq(a32.F, amix.F) || !same_sell(at32.h, atmix.h) ||
        !same_freq(at32.F, atmix.F))
        fail("FP64 input in the FP32 form");

    // 3. every entry recovered from each orientation
    if (!same_entries(recover(a32, ld, m), entries_of(n, rp.data(), ci.data(), vf.data())))
        fail("A: entries recovered from the layouts");
    if (!same_entries(recover(at32, ld, n), entries_of(m, cp.data(), ri.data(), cv.data())))
        fail("A^T: entries recovered from the layouts");
    if (a32.h.nnz + a32.F.t[0].nnz + a32.F.t[1].nnz != nnz) fail("A: entry count");
    if (at32.h.nnz + at32.F.t[0].nnz + at32.F.t[1].nnz != nnz) fail("A^T: entry count");

    std::printf("%s: nnz %lld, A h=%d (h1=%d, tiers %lld+%lld), A^T h=%d (h1=%d, tiers %lld+%lld), "
                "pad %d: %s\n",
                pre.c_str(), (long long)nnz, a32.F.h, a32.F.h1, (long long)a32.F.t[0].nnz,
                (long long)a32.F.t[1].nnz, at32.F.h, at32.F.h1, (long long)at32.F.t[0].nnz,
                (long long)at32.F.t[1].nnz, freq_pad(ld), g_fail ? "FAILED" : "ok");
    return g_fail ? 1 : 0;
}
