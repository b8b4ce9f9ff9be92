// k_select.cu -- the enforcement step of Alg. 2 (steps 2 and 4): find, per
// column (Sec. 4) or over the whole factor (Alg. 2 as printed), the value of
// the t-th largest positive entry, with ties to the lower index.  The
// survivors are written afterwards, row by row and in column order, by the
// emit kernel (or, for a caller's dense buffer, by apply_thresholds).
//
// Input: the projected candidate X in column-major order (Xt[c*ldx+i],
// rows i < rows, every entry >= +0).  For non-negative IEEE numbers the bit
// pattern read as an unsigned integer orders exactly like the value, so the
// threshold is found by radix selection on the bit patterns:
//   pass 1  an 11-bit histogram of the top bits (FP32: exponent and the
//           first 3 mantissa bits, 8 buckets per binade; FP64: exponent),
//   pass 2  the entries of the bucket holding the t-th largest value are
//           copied to a candidate list in shared memory,
//   then    the remaining bits are resolved by radix rounds over the
//           candidates only, and ties by a radix select over their indices.
// When it marks survivors (FP32 form, column mode) one CTA of 1024 threads
// owns a column and starts from a hint, the column's threshold of the
// previous selection: one pass counts and marks the entries above the three
// bins around the hint and lists the entries in them; when the t-th largest
// is among those, passes 1 and 2 are skipped (rounds over the list only),
// otherwise the marks are taken back and the search runs as above.
// Otherwise a thread-block cluster of up to two CTAs owns a column (or the
// whole matrix); the CTAs add their histograms through distributed shared
// memory.  Every CTA reads its slice of the column straight from global
// memory (the candidate was just written, so it is in the L2) with 16-byte
// loads; shared memory holds only the histogram and the candidate list.  If
// a CTA's candidates overflow its list, the bucket is resolved with passes
// over the data instead (same result, slower).
//
// Output per segment s (column, or 0 in matrix mode): tau[s] (bit pattern)
// and cut[s]: an entry survives iff it is positive and its bits are > tau,
// or == tau and its index (row, or row-major i*k+c in matrix mode) is
// <= cut.  tau = 0 keeps every positive entry; tau = all ones keeps none.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace espnmf {

constexpr int kSelThreads = 1024;
constexpr int kSelMaxCluster = 2;
constexpr int kSelMaxClusterWhole = 8;   // one segment (matrix mode): a portable cluster

template <typename T> struct Vec4Of;
template <> struct Vec4Of<float> { using type = float4; };
struct alignas(16) Double4x { double2 a, b; };
template <> struct Vec4Of<double> { using type = Double4x; };
constexpr int kHist = 2048;
constexpr int kCandCap = 12288;  // candidates per CTA
constexpr size_t kSelSmemMax = 210 * 1024;

template <typename T>
struct SelSmem {
    using K = typename KeyBits<T>::K;
    static constexpr size_t hist = 0;
    static constexpr size_t misc = hist + kHist * 4;   // 512 B of scan scratch
    static constexpr size_t ckey = misc + 512;
    static constexpr size_t cidx = ckey + (size_t)kCandCap * sizeof(K);
    static constexpr size_t data = (cidx + (size_t)kCandCap * 4 + 15) & ~(size_t)15;
};

struct ScanOut {
    int bin;
    unsigned long long before;   // count in the bins scanned before `bin`
    unsigned long long total;
    unsigned long long count;    // count in `bin`
};

// Adds the cluster's histograms (first nb bins, kBinsPerThread per thread)
// and finds the bin where the running count -- from the top when
// `descending` -- reaches `need`.  Every CTA computes the same result.
constexpr int kBinsPerThread = kHist / kSelThreads;

__device__ ScanOut cluster_scan(cg::cluster_group& cluster, unsigned* hist, int nb,
                                unsigned long long need, bool descending,
                                unsigned long long* wsum, unsigned long long* res)
{
    const int C = (int)cluster.num_blocks();
    // every CTA's histogram is complete (a block barrier for a lone CTA)
    if (C > 1) cluster.sync();
    else __syncthreads();
    const int tid = threadIdx.x;
    unsigned long long v[kBinsPerThread];
#pragma unroll
    for (int u = 0; u < kBinsPerThread; ++u) {
        v[u] = 0;
        const int o = tid * kBinsPerThread + u;
        if (o < nb) {
            const int b = descending ? nb - 1 - o : o;
            for (int r = 0; r < C; ++r) v[u] += cluster.map_shared_rank(hist, r)[b];
        }
    }
    if (C > 1) cluster.sync();   // remote reads done: histograms may be reused
    unsigned long long local = 0;
#pragma unroll
    for (int u = 0; u < kBinsPerThread; ++u) local += v[u];
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    unsigned long long incl = local;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long x = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long x = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += x;
        }
        if (lane < nw) wsum[lane] = w;
    }
    if (tid == 0) {
        res[0] = ~0ull;
        res[1] = 0;
        res[2] = 0;
    }
    __syncthreads();
    const unsigned long long start = (warp > 0 ? wsum[warp - 1] : 0) + incl - local;
    const unsigned long long total = wsum[nw - 1];
    if (start < need && start + local >= need) {
        unsigned long long cum = start;
#pragma unroll
        for (int u = 0; u < kBinsPerThread; ++u) {
            if (cum + v[u] >= need) {
                const int o = tid * kBinsPerThread + u;
                res[0] = (unsigned long long)(descending ? nb - 1 - o : o);
                res[1] = cum;
                res[2] = v[u];
                break;
            }
            cum += v[u];
        }
    }
    __syncthreads();
    ScanOut r;
    r.bin = (int)res[0];
    r.before = res[1];
    r.count = res[2];
    r.total = total;
    __syncthreads();
    return r;
}

// For a positive FP32 bit pattern: the integer mantissa m (implicit bit
// included) and the exponent s with x = m 2^s.
__device__ __forceinline__ unsigned long long mantissa24(uint32_t key)
{
    const uint32_t e = (key >> 23) & 0xffu;
    return (unsigned long long)((key & 0x7fffffu) | (e ? 0x800000u : 0u));
}
__device__ __forceinline__ int exponent_of(uint32_t key)
{
    const int e = (int)((key >> 23) & 0xffu);
    return e ? e - 150 : -149;
}

// Optional survivor marking (COLUMN mode): once a column's threshold is
// known, each CTA walks its slice again, sets bit (c % 32) of word c / 32 of
// row i in rowbits ([rows][mark_words]) for every survivor and writes the
// sum of the survivors' squares (the column's diagonal entry of F^T F, as a
// compensated FP32 pair, fixed order) to diag_part[c * clusterDim + rank].
struct SelMark {
    uint32_t* rowbits = nullptr;
    int words = 0;
    double* diag_part = nullptr;
    void* hint = nullptr;   // [k] keys: the last threshold of each column (0: none)
    unsigned long long* counts = nullptr;   // [2]: warm starts that held, full searches
};

template <typename T>
__global__ void __launch_bounds__(kSelThreads)
select_kernel(const T* __restrict__ Xt, int64_t ldx, int64_t rows, int k,
              int64_t t, int mode, typename KeyBits<T>::K* __restrict__ tau_out,
              uint32_t* __restrict__ cut_out, SelMark mark)
{
    using K = typename KeyBits<T>::K;
    constexpr int TS = KeyBits<T>::top_shift;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ DFloat wsq[kSelThreads / 32];
    __shared__ unsigned long long wisq[kSelThreads / 32], wisq1[kSelThreads / 32];
    __shared__ double bucket_sq;   // the bucket survivors' exact sum of squares
    __shared__ unsigned long long s_above;   // warm start: entries above the window
    unsigned* hist = reinterpret_cast<unsigned*>(smem_raw + SelSmem<T>::hist);
    unsigned long long* wsum = reinterpret_cast<unsigned long long*>(smem_raw + SelSmem<T>::misc);
    unsigned long long* res = wsum + 32;
    unsigned* ccount = reinterpret_cast<unsigned*>(res + 3);
    K* ckey = reinterpret_cast<K*>(smem_raw + SelSmem<T>::ckey);
    uint32_t* cidx = reinterpret_cast<uint32_t*>(smem_raw + SelSmem<T>::cidx);

    const int C = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int seg = blockIdx.y;
    const bool matrix = mode == TOPT_MATRIX;
    const int64_t seg_len = matrix ? (int64_t)k * rows : rows;
    int64_t per = (seg_len + C - 1) / C;
    per = (per + 3) & ~(int64_t)3;
    const int64_t lo = (int64_t)crank * per < seg_len ? (int64_t)crank * per : seg_len;
    const int64_t hi = lo + per < seg_len ? lo + per : seg_len;
    const int nloc = (int)(hi - lo);
    const int tid = threadIdx.x;
    auto addr = [&](int64_t g) -> int64_t {
        if (!matrix) return (int64_t)seg * ldx + g;
        const int64_t c = g / rows;
        return c * ldx + (g - c * rows);
    };
    auto index_of = [&](int e) -> uint32_t {
        const int64_t g = lo + e;
        if (!matrix) return (uint32_t)g;
        const int64_t c = g / rows, i = g - c * rows;
        return (uint32_t)(i * k + c);
    };

    // t = 0 keeps nothing; mode NONE keeps every positive entry
    if (mode == TOPT_NONE || t <= 0) {
        if (crank == 0 && tid == 0) {
            tau_out[seg] = mode == TOPT_NONE ? (K)0 : ~(K)0;
            cut_out[seg] = 0xffffffffu;
        }
        if (mark.rowbits && tid == 0) mark.diag_part[(size_t)seg * C + crank] = 0.0;
        return;
    }
    // visits this CTA's entries with their keys: 16-byte loads (four in
    // flight per thread) of the contiguous slice of a column; strided
    // addressing in matrix mode.  The loop bound is uniform across a warp,
    // so fn may use warp collectives; `ok` marks lanes holding an entry.
    using V4 = typename Vec4Of<T>::type;
    auto for_each = [&](auto&& fn) {
        if (!matrix) {
            const T* src = Xt + (int64_t)seg * ldx + lo;
            const V4* s4 = reinterpret_cast<const V4*>(src);
            const int nv = nloc / 4;
            const int span = (int)blockDim.x * 4;
            const int nround = (nv + span - 1) / span * span;
            for (int q0 = tid; q0 < nround; q0 += span) {
                V4 v[4];
                bool in[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * (int)blockDim.x;
                    in[u] = q < nv;
                    if (in[u]) v[u] = s4[q];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u * (int)blockDim.x;
                    const T* x = reinterpret_cast<const T*>(&v[u]);
#pragma unroll
                    for (int w = 0; w < 4; ++w) fn(in[u] ? KeyBits<T>::of(x[w]) : (K)0, 4 * q + w, in[u]);
                }
            }
            // tail (fewer than 4 entries), the same for every warp's lanes
            const int tail = nloc - nv * 4;
            if (tail > 0) {
                const bool in = tid < tail;
                const int e = nv * 4 + (in ? tid : 0);
                fn(in ? KeyBits<T>::of(src[e]) : (K)0, e, in);
            }
        } else {
            const int nround = (nloc + (int)blockDim.x - 1) / (int)blockDim.x * (int)blockDim.x;
            for (int e0 = 0; e0 < nround; e0 += blockDim.x) {
                const int e = e0 + tid;
                const bool in = e < nloc;
                fn(in ? KeyBits<T>::of(Xt[addr(lo + e)]) : (K)0, e, in);
            }
        }
    };
    auto key_at = [&](int e) -> K { return KeyBits<T>::of(Xt[addr(lo + e)]); };
    if (tid == 0) bucket_sq = 0.0;   // read by mark_finish after barriers
    // Survivor marking (column mode): a survivor sets its row's bit and
    // adds its square to this thread's FP64 sum (msq); mark_finish reduces
    // the sums in a fixed order into the column's diagonal partial.
    DFloat msq;   // compensated FP32 (only FP32 contexts mark)
    const uint32_t mbit = 1u << (seg & 31);
    auto mark_one = [&](K key, uint32_t row) {
        if (!ESPNMF_CHECK((int64_t)row < rows, CHK_CAND_ROW)) return;
        atomicOr(mark.rowbits + (seg >> 5) + (size_t)row * mark.words, mbit);
        const float x = (float)KeyBits<T>::value(key);
        df_add_prod(msq, x, x);
    };
    auto mark_finish = [&]() {
        const DFloat sq = df_warp_sum(msq);
        if ((tid & 31) == 0) wsq[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            DFloat tot;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(tot, wsq[w].hi, wsq[w].lo);
            if (bucket_sq != 0.0) {
                const float bh = (float)bucket_sq;
                df_add(tot, bh, (float)(bucket_sq - (double)bh));
            }
            reinterpret_cast<float2*>(mark.diag_part)[(size_t)seg * C + crank] = make_float2(tot.hi, tot.lo);
        }
    };
    // every positive entry survives (at most t of them)
    auto mark_all = [&]() {
        for_each([&](K key, int e, bool in) {
            if (in && key != 0) mark_one(key, (uint32_t)(lo + e));
        });
        mark_finish();
    };

    const int lane = tid & 31;
    const bool marking = mark.rowbits != nullptr;
    K* hint = static_cast<K*>(mark.hint);
    constexpr int KB = (int)(8 * sizeof(K));
    // the first histogram's bin of a positive key
    auto bucket_of = [&](K key) -> int { return (int)((key >> TS) & (K)(kHist - 1)); };
    // appends this lane's entry to the candidate list (warp-aggregated)
    auto append = [&](bool hit, K key, int e) {
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m == 0u) return;
        unsigned base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(ccount, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (hit) {
            const unsigned pos = base + (unsigned)__popc(m & ((1u << lane) - 1u));
            if (pos < (unsigned)kCandCap) {
                ckey[pos] = key;
                cidx[pos] = index_of(e);
            }
        }
    };

    unsigned long long need = (unsigned long long)t;
    K prefix = 0;
    int shift = 0;     // bits below `shift` are still open
    int nc = 0;
    bool use_list = true;
    int base_bucket = 0;   // lowest first-histogram bin among the candidates
    bool warm = false;

    // ---- warm start (column mode): the threshold of the previous selection
    // of this column names a first-histogram bin; one pass counts the
    // entries above that bin's neighbours and lists the entries of the
    // three bins (each CTA of the column's cluster over its own part, the
    // counts then summed over the cluster).  If the t-th largest lies among
    // them, the first histogram and its pass are not needed; otherwise the
    // marks set above the window are taken back and the full search follows.
    if (hint != nullptr && !matrix) {
        const K h = hint[seg];
        if (h != (K)0 && h != ~(K)0) {
            const int hb = bucket_of(h);
            const int lo_b = hb > 0 ? hb - 1 : 0, hi_b = hb < kHist - 1 ? hb + 1 : kHist - 1;
            if (tid == 0) {
                *ccount = 0;
                s_above = 0;
            }
            __syncthreads();
            // the window in key space: [lo_key, hi_key], lo_key > 0
            const K lo_key = lo_b > 0 ? (K)lo_b << TS : (K)1;
            const K hi_key = (((K)hi_b + 1) << TS) - 1;
            unsigned above = 0;
            if (!matrix) {
                // sixteen entries per thread per round (four 16-byte loads);
                // the round's hits are placed by one warp scan
                using V4 = typename Vec4Of<T>::type;
                const V4* s4 = reinterpret_cast<const V4*>(Xt + (int64_t)seg * ldx + lo);
                const int nv = nloc / 4;
                const int span = (int)blockDim.x * 4;
                const int nround = (nv + span - 1) / span * span;
                for (int q0 = tid; q0 < nround; q0 += span) {
                    K keys[16];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u * (int)blockDim.x;
                        V4 v;
                        if (q < nv) v = s4[q];
                        const T* x = reinterpret_cast<const T*>(&v);
#pragma unroll
                        for (int w = 0; w < 4; ++w) keys[4 * u + w] = q < nv ? KeyBits<T>::of(x[w]) : (K)0;
                    }
                    unsigned hm = 0;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const K key = keys[j];
                        if (key > hi_key) {
                            ++above;
                            if (marking) {
                                const int e = 4 * (q0 + (j >> 2) * (int)blockDim.x) + (j & 3);
                                mark_one(key, (uint32_t)(lo + e));
                            }
                        }
                        if (key >= lo_key && key <= hi_key) hm |= 1u << j;
                    }
                    const unsigned nh = (unsigned)__popc(hm);
                    unsigned incl = nh;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const unsigned y = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += y;
                    }
                    unsigned base = 0;
                    if (lane == 31 && incl) base = atomicAdd(ccount, incl);
                    base = __shfl_sync(0xffffffffu, base, 31) + incl - nh;
                    if (hm) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if ((hm >> j) & 1u) {
                                if (base < (unsigned)kCandCap) {
                                    ckey[base] = keys[j];
                                    cidx[base] = (uint32_t)(lo + 4 * (q0 + (j >> 2) * (int)blockDim.x) + (j & 3));
                                }
                                ++base;
                            }
                        }
                    }
                }
                // tail (fewer than 4 entries)
                const int tail = nloc - nv * 4;
                if (tail > 0) {
                    const bool in = tid < tail;
                    const int e = nv * 4 + (in ? tid : 0);
                    const K key = in ? KeyBits<T>::of(Xt[(int64_t)seg * ldx + lo + e]) : (K)0;
                    if (key > hi_key) {
                        ++above;
                        if (marking) mark_one(key, (uint32_t)(lo + e));
                    }
                    append(key >= lo_key && key <= hi_key, key, e);
                }
            }
            above = __reduce_add_sync(0xffffffffu, above);
            if (lane == 0 && above) atomicAdd(&s_above, (unsigned long long)above);
            __syncthreads();
            const unsigned long long nca = *ccount;
            unsigned long long ab = s_above, nca_all = nca;
            bool overflow = nca > (unsigned long long)kCandCap;
            __syncthreads();
            if (C > 1) {
                // the cluster's totals: each CTA publishes its two counts
                // (below 2^32: a CTA holds fewer entries) in its histogram
                if (tid == 0) {
                    hist[0] = (unsigned)ab;
                    hist[1] = (unsigned)nca;
                }
                cluster.sync();
                ab = 0;
                nca_all = 0;
                overflow = false;
                for (int r = 0; r < C; ++r) {
                    const unsigned* hr = cluster.map_shared_rank(hist, r);
                    ab += hr[0];
                    nca_all += hr[1];
                    overflow = overflow || hr[1] > (unsigned)kCandCap;
                }
                cluster.sync();   // remote reads done: the histograms may be reused
            }
            if (!overflow && ab < need && ab + nca_all >= need) {
                warm = true;
                need -= ab;
                prefix = 0;
                shift = TS + 11;   // the candidates still differ in their bin
                nc = (int)nca;
                base_bucket = lo_b;
            } else if (marking) {
                for_each([&](K key, int e, bool in) {
                    if (in && key > hi_key)
                        atomicAnd(mark.rowbits + (seg >> 5) + (size_t)(lo + e) * mark.words, ~mbit);
                });
                msq = DFloat();
                __syncthreads();
            }
        }
    }

    if (hint != nullptr && mark.counts != nullptr && tid == 0 && crank == 0)
        atomicAdd(mark.counts + (warm ? 0 : 1), 1ull);
    if (!warm) {
        // ---- pass 1: histogram of the top 11 bits of the positive entries
        for (int b = tid; b < kHist; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for_each([&](K key, int, bool in) {
            if (in && key != 0) atomicAdd(&hist[bucket_of(key)], 1u);
        });
        __syncthreads();
        const ScanOut s1 = cluster_scan(cluster, hist, kHist, need, true, wsum, res);
        if (s1.total <= need) {   // at most t positive entries: keep them all
            if (crank == 0 && tid == 0) {
                tau_out[seg] = 0;
                cut_out[seg] = 0xffffffffu;
                if (hint) hint[seg] = 0;
            }
            if (marking) mark_all();
            return;
        }
        need -= s1.before;
        prefix = (K)s1.bin << TS;
        shift = TS;
        base_bucket = s1.bin;

        // ---- pass 2: the bucket's entries into the candidate list
        if (tid == 0) *ccount = 0;
        __syncthreads();
        for_each([&](K key, int e, bool in) {
            const bool hit = in && key != 0 && (key >> shift) == (prefix >> shift);
            // above the threshold's bucket: a survivor whatever the threshold
            if (marking && in && (key >> shift) > (prefix >> shift)) mark_one(key, (uint32_t)(lo + e));
            append(hit, key, e);
        });
        __syncthreads();
        const unsigned ncand = *ccount;
        __syncthreads();
        if (C > 1) {
            if (tid == 0) hist[0] = ncand > (unsigned)kCandCap ? 1u : 0u;
            __syncthreads();
            const ScanOut ov = cluster_scan(cluster, hist, 1, 1, false, wsum, res);
            use_list = ov.total == 0;   // no CTA overflowed
        } else {
            use_list = ncand <= (unsigned)kCandCap;
        }
        nc = use_list ? (int)ncand : 0;
    }

    // ---- the remaining bits: radix rounds of up to 11 bits; the last
    // round's bin holds exactly the entries equal to the threshold
    unsigned long long eq = 0;
    while (shift > 0) {
        const int bits = shift >= 11 ? 11 : shift;
        const int sh = shift - bits;
        const unsigned mask = (1u << bits) - 1u;
        // (key >> shift) == (prefix >> shift), for shift < KB
        auto open = [&](K key) { return shift >= KB || (key >> shift) == (prefix >> shift); };
        for (int b = tid; b < kHist; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        if (use_list) {
            for (int q = tid; q < nc; q += blockDim.x) {
                const K key = ckey[q];
                if (open(key)) atomicAdd(&hist[(unsigned)(key >> sh) & mask], 1u);
            }
        } else {
            for (int e = tid; e < nloc; e += blockDim.x) {
                const K key = key_at(e);
                if (key != 0 && open(key)) atomicAdd(&hist[(unsigned)(key >> sh) & mask], 1u);
            }
        }
        __syncthreads();
        const ScanOut sr = cluster_scan(cluster, hist, 1 << bits, need, true, wsum, res);
        need -= sr.before;
        prefix |= (K)sr.bin << sh;
        shift = sh;
        eq = sr.count;
    }
    const K tau = prefix;
    uint32_t cut = 0xffffffffu;
    if (need < eq) {
        // keep the `need` smallest indices among the ties: radix select on
        // the index, ascending, 11 bits at a time
        uint32_t ipre = 0;
        int ish = 32;
        while (ish > 0) {
            const int bits = ish >= 11 ? 11 : ish;
            const int sh = ish - bits;
            const unsigned mask = (1u << bits) - 1u;
            for (int b = tid; b < kHist; b += blockDim.x) hist[b] = 0;
            __syncthreads();
            auto consider = [&](K key, uint32_t ix) {
                if (key == tau && (ish >= 32 || (ix >> ish) == (ipre >> ish)))
                    atomicAdd(&hist[(ix >> sh) & mask], 1u);
            };
            if (use_list) {
                for (int q = tid; q < nc; q += blockDim.x) consider(ckey[q], cidx[q]);
            } else {
                for (int e = tid; e < nloc; e += blockDim.x) consider(key_at(e), index_of(e));
            }
            __syncthreads();
            const ScanOut si = cluster_scan(cluster, hist, 1 << bits, need, false, wsum, res);
            need -= si.before;
            ipre |= (uint32_t)si.bin << sh;
            ish = sh;
        }
        cut = ipre;
    }
    if (crank == 0 && tid == 0) {
        tau_out[seg] = tau;
        cut_out[seg] = cut;
        if (hint) hint[seg] = tau;
    }
    if (marking) {
        // the survivors inside the bucket: from the candidate list, or by a
        // pass over the slice if a CTA's list overflowed
        const K bucket = prefix >> TS;   // the first histogram's bin
        if (use_list) {
            // The list's order depends on the order of the appends, so its
            // survivors' squares are added exactly: an entry is x = m 2^s
            // with an integer m < 2^24, the candidates' bins (one, or three
            // after a warm start) span at most two exponents s0 and s0 + 1,
            // and sum(m^2) per exponent fits 64 bits (at most kCandCap terms).
            const int s0 = exponent_of((uint32_t)((K)base_bucket << TS));
            unsigned long long isq0 = 0, isq1 = 0;
            for (int q = tid; q < nc; q += blockDim.x) {
                if (keep_entry<T>(KeyBits<T>::value(ckey[q]), tau, cut, cidx[q]) &&
                    ESPNMF_CHECK((int64_t)cidx[q] < rows, CHK_CAND_ROW)) {
                    atomicOr(mark.rowbits + (seg >> 5) + (size_t)cidx[q] * mark.words, mbit);
                    const unsigned long long m = mantissa24((uint32_t)ckey[q]);
                    if (exponent_of((uint32_t)ckey[q]) == s0) isq0 += m * m;
                    else isq1 += m * m;
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                isq0 += __shfl_xor_sync(0xffffffffu, isq0, off);
                isq1 += __shfl_xor_sync(0xffffffffu, isq1, off);
            }
            if ((tid & 31) == 0) {
                wisq[tid >> 5] = isq0;
                wisq1[tid >> 5] = isq1;
            }
            __syncthreads();
            if (tid == 0) {
                unsigned long long t0 = 0, t1 = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    t0 += wisq[w];
                    t1 += wisq1[w];
                }
                bucket_sq = ldexp((double)t0, 2 * s0) + ldexp((double)t1, 2 * s0 + 2);
            }
        } else {
            for_each([&](K key, int e, bool in) {
                if (in && key != 0 && (key >> TS) == bucket &&
                    keep_entry<T>(KeyBits<T>::value(key), tau, cut, (uint32_t)(lo + e)))
                    mark_one(key, (uint32_t)(lo + e));
            });
        }
        mark_finish();
    }
}

// CTAs per cluster: about two CTAs per SM over all segments, at most
// kSelMaxCluster per column (larger clusters measured slower with k columns
// in flight) and kSelMaxClusterWhole for the single segment of matrix mode
// (the whole factor), at least 2048 entries per CTA.  When it marks
// survivors (column mode) the cluster size is a fixed function of the
// column length (it decides how the Gram diagonal's partial sums are
// grouped, so it must not depend on timing): two CTAs for columns of at
// least kSelMarkSplitRows entries, else one.
constexpr int64_t kSelMarkSplitRows = 32768;
static int sel_cluster(int64_t rows, int k, int mode, int sm_count, bool marking)
{
    if (marking && mode == TOPT_COLUMN) return rows >= kSelMarkSplitRows ? 2 : 1;
    const int nseg = mode == TOPT_MATRIX ? 1 : k;
    const int64_t seg_len = mode == TOPT_MATRIX ? (int64_t)k * rows : rows;
    int C = (int)((2 * (int64_t)sm_count + nseg - 1) / nseg);
    const int cap = nseg == 1 ? kSelMaxClusterWhole : kSelMaxCluster;
    if (C > cap) C = cap;
    const int64_t by_len = (seg_len + 2047) / 2048;
    if (C > by_len) C = (int)by_len;
    if (C < 1) C = 1;
    return C;
}

template <typename T>
cudaError_t launch_select(const T* Xt, int64_t ldx, int64_t rows, int k,
                          int64_t t, int mode, void* tau, uint32_t* cut,
                          cudaStream_t st, int sm_count, uint32_t* rowbits,
                          double* diag_part, void* hint, unsigned long long* counts)
{
    if (rows == 0) return cudaSuccess;
    const int nseg = mode == TOPT_MATRIX ? 1 : k;
    const bool marking = rowbits != nullptr && mode == TOPT_COLUMN;
    const int C = sel_cluster(rows, k, mode, sm_count, marking);
    const size_t smem = SelSmem<T>::data;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, (unsigned)nseg, 1);
    cfg.blockDim = dim3(kSelThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    using K = typename KeyBits<T>::K;
    SelMark mark;
    if (marking) {
        mark.rowbits = rowbits;
        mark.words = (k + 31) / 32;
        mark.diag_part = diag_part;
        mark.hint = hint;
        mark.counts = counts;
    }
    return cudaLaunchKernelEx(&cfg, select_kernel<T>, Xt, ldx, rows, k, t, mode,
                              static_cast<K*>(tau), cut, mark);
}

// Cluster size launch_select uses when marking for k columns of `rows`
// entries (the number of diagonal partials per column it writes).
int select_cluster(int64_t rows, int k, int mode, int sm_count)
{
    return sel_cluster(rows, k, mode, sm_count, true);
}

ESPNMF_CHECK_READER(check_flags_select)

// In-place projection + enforcement of a caller's dense rows x k buffer
// (leading dimension ld) with thresholds from select_kernel.
template <typename T>
__global__ void apply_thresholds_kernel(T* X, int64_t rows, int k, int64_t ld, int mode,
                                        const typename KeyBits<T>::K* __restrict__ tau,
                                        const uint32_t* __restrict__ cut, unsigned* status)
{
    // a non-finite entry was already seen (by the column-major copy that
    // feeds the selector): X is left as the caller gave it
    if (*reinterpret_cast<volatile unsigned*>(status) & ST_NONFINITE) return;
    bool bad = false;
    const int64_t total = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int c = (int)(e - r * k);
        const T x = X[r * ld + c];
        if (!isfinite((double)x)) bad = true;
        const T v = x > T(0) ? x : T(0);
        const int s = mode == TOPT_MATRIX ? 0 : c;
        const uint32_t ix = mode == TOPT_MATRIX ? (uint32_t)(r * k + c) : (uint32_t)r;
        X[r * ld + c] = keep_entry<T>(v, tau[s], cut[s], ix) ? v : T(0);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

template <typename T>
cudaError_t launch_apply_thresholds(T* X, int64_t rows, int k, int64_t ld, int mode,
                                    const void* tau, const uint32_t* cut, unsigned* status,
                                    cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    int64_t grid = (rows * k + 255) / 256;
    if (grid > 65535) grid = 65535;
    using K = typename KeyBits<T>::K;
    apply_thresholds_kernel<T><<<(unsigned)grid, 256, 0, st>>>(
        X, rows, k, ld, mode, static_cast<const K*>(tau), cut, status);
    return cudaGetLastError();
}

cudaError_t setup_select()
{
    cudaError_t e = cudaFuncSetAttribute(select_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSelSmemMax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(select_kernel<double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSelSmemMax);
}

template cudaError_t launch_select<float>(const float*, int64_t, int64_t, int, int64_t, int, void*, uint32_t*, cudaStream_t, int, uint32_t*, double*, void*, unsigned long long*);
template cudaError_t launch_select<double>(const double*, int64_t, int64_t, int, int64_t, int, void*, uint32_t*, cudaStream_t, int, uint32_t*, double*, void*, unsigned long long*);
template cudaError_t launch_apply_thresholds<float>(float*, int64_t, int, int64_t, int, const void*, const uint32_t*, unsigned*, cudaStream_t);
template cudaError_t launch_apply_thresholds<double>(double*, int64_t, int, int64_t, int, const void*, const uint32_t*, unsigned*, cudaStream_t);

}  // namespace espnmf
