// k_select.cu -- the enforcement step of Alg. 2 (steps 2 and 4): keep only
// the t largest positive entries of every column (Sec. 4) or of the whole
// factor (Alg. 2 as printed), ties to the lower index.
//
// Input is the projected candidate X in column-major order (Xt[c*ldx+i],
// rows i < rows, every entry >= +0).  For non-negative IEEE numbers the bit pattern read
// as an unsigned integer orders exactly like the value, so the t-th largest
// value is found by an MSB-first radix select over the bit patterns: 8 bits
// per round, 4 rounds for FP32 and 8 for FP64.
//
// One thread-block cluster (up to 8 CTAs) owns a column (or the whole
// matrix).  Each CTA owns a contiguous slice of it, kept in shared memory
// when it fits, and builds a 256-bin histogram per round with warp-
// aggregated shared-memory atomics; the cluster adds its CTAs' histograms
// through distributed shared memory, and every CTA then picks the same
// digit.  When more entries equal the threshold than may be kept, a second
// radix select over their indices finds the cut-off index, so exactly
// min(t, #positive) entries survive.  Survivors are appended to their row of
// the row-packed factor (row counter atomics; pair order inside a row is
// irrelevant to every consumer).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace espnmf {

constexpr int kSelThreads = 512;
constexpr int kSelWarps = kSelThreads / 32;
constexpr size_t kSelFixedSmem = (size_t)(kSelWarps * 256 + 2 * 256 + 256) * 4 + 64;
constexpr size_t kSelSmemMax = 200 * 1024;

template <typename T> struct Bits;
template <> struct Bits<float> {
    using K = uint32_t;
    static constexpr int nbits = 32;
    __device__ static K of(float x) { return __float_as_uint(x); }
};
template <> struct Bits<double> {
    using K = unsigned long long;
    static constexpr int nbits = 64;
    __device__ static K of(double x) { return (K)__double_as_longlong(x); }
};

struct SelShared {
    unsigned* whist;   // [kSelWarps][256]
    unsigned* bhist;   // [2][256], read by the other CTAs of the cluster
    unsigned* hsum;    // [256] cluster totals
    unsigned long long* bcast;  // [4] results of the digit scan
};

// All 32 lanes call this with the same trip count.
__device__ __forceinline__ void hist_add(unsigned* wh, unsigned digit, bool valid)
{
    const unsigned key = valid ? digit : 0x100u;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&wh[digit], (unsigned)__popc(peers));
}

// Sums the warp histograms into bhist[buf], adds the cluster's CTAs into
// hsum.  Ends with hsum visible to the whole CTA.
__device__ void cluster_hist_total(cg::cluster_group& cluster, SelShared& S, int buf)
{
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        unsigned s = 0;
        for (int w = 0; w < kSelWarps; ++w) s += S.whist[w * 256 + b];
        S.bhist[buf * 256 + b] = s;
    }
    cluster.sync();
    const int C = (int)cluster.num_blocks();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        unsigned s = 0;
        for (int r = 0; r < C; ++r) {
            const unsigned* rem = cluster.map_shared_rank(S.bhist + buf * 256, r);
            s += rem[b];
        }
        S.hsum[b] = s;
    }
    for (int e = threadIdx.x; e < kSelWarps * 256; e += blockDim.x) S.whist[e] = 0;
    __syncthreads();
}

// Finds, walking the bins from the top (descending) or the bottom, the bin
// where the running count reaches `need`.  Writes bcast[0] = bin,
// bcast[1] = count before that bin, bcast[2] = total of all bins.
__device__ void scan_bins(SelShared& S, unsigned long long need, bool descending)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long local = 0;
        for (int j = 0; j < 8; ++j) {
            const int o = lane * 8 + j;
            const int b = descending ? 255 - o : o;
            local += S.hsum[b];
        }
        unsigned long long incl = local;
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned hit = __ballot_sync(0xffffffffu, incl >= need);
        if (lane == 0) S.bcast[2] = total;
        if (hit != 0 && lane == __ffs(hit) - 1) {
            unsigned long long cum = incl - local;
            for (int j = 0; j < 8; ++j) {
                const int o = lane * 8 + j;
                const int b = descending ? 255 - o : o;
                if (cum + S.hsum[b] >= need) {
                    S.bcast[0] = (unsigned long long)b;
                    S.bcast[1] = cum;
                    break;
                }
                cum += S.hsum[b];
            }
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads)
select_kernel(const T* __restrict__ Xt, int64_t ldx, int64_t rows, int k,
              int64_t t, int mode, int32_t* __restrict__ cnt,
              int32_t* __restrict__ colo, T* __restrict__ valo,
              int64_t cache_elems, unsigned* status, int ld)
{
    using K = typename Bits<T>::K;
    constexpr int NB = Bits<T>::nbits;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SelShared S;
    S.whist = reinterpret_cast<unsigned*>(smem_raw);
    S.bhist = S.whist + kSelWarps * 256;
    S.hsum = S.bhist + 2 * 256;
    S.bcast = reinterpret_cast<unsigned long long*>(S.hsum + 256);
    T* cache = reinterpret_cast<T*>(smem_raw + kSelFixedSmem);

    const int C = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int seg = blockIdx.y;
    const bool matrix = mode == TOPT_MATRIX;
    // Segment positions g in [0, seg_len): column mode g = row of column
    // `seg`; matrix mode g = c * rows + i over all columns.
    const int64_t seg_len = matrix ? (int64_t)k * rows : rows;
    int64_t per = (seg_len + C - 1) / C;
    per = (per + 3) & ~(int64_t)3;
    const int64_t lo = (int64_t)crank * per < seg_len ? (int64_t)crank * per : seg_len;
    const int64_t hi = lo + per < seg_len ? lo + per : seg_len;
    const int64_t nloc = hi - lo;
    const bool cached = nloc <= cache_elems;
    const int tid = threadIdx.x;
    auto addr = [&](int64_t g) -> int64_t {
        if (!matrix) return (int64_t)seg * ldx + g;
        const int64_t c = g / rows;
        return c * ldx + (g - c * rows);
    };

    for (int e = tid; e < kSelWarps * 256; e += blockDim.x) S.whist[e] = 0;
    if (cached)
        for (int64_t e = tid; e < nloc; e += blockDim.x) cache[e] = Xt[addr(lo + e)];
    __syncthreads();

    auto value = [&](int64_t e) -> T { return cached ? cache[e] : Xt[addr(lo + e)]; };
    // index used for ties: the row (column mode) or the row-major i*k+c
    auto tie_index = [&](int64_t e) -> uint32_t {
        const int64_t g = lo + e;
        if (!matrix) return (uint32_t)g;
        const int64_t c = g / rows, i = g - c * rows;
        return (uint32_t)(i * k + c);
    };
    unsigned* wh = S.whist + (tid >> 5) * 256;
    const int64_t trip = (nloc + blockDim.x - 1) / blockDim.x * blockDim.x;

    K tau = 0;                      // keep key > tau, or key == tau and index <= cut
    uint32_t cut = 0xffffffffu;
    bool keep_none = t <= 0 && mode != TOPT_NONE;
    int buf = 0;

    if (!keep_none && mode != TOPT_NONE) {
        // Round 0 also counts the positive entries.
        unsigned long long need = (unsigned long long)t;
        K prefix = 0;
        bool all = false;
        unsigned long long last_bin_count = 0;
        for (int shift = NB - 8; shift >= 0; shift -= 8) {
            for (int64_t e0 = 0; e0 < trip; e0 += blockDim.x) {
                const int64_t e = e0 + tid;
                bool ok = false;
                unsigned d = 0;
                if (e < nloc) {
                    const K key = Bits<T>::of(value(e));
                    const bool match = shift == NB - 8 ? true : ((key ^ prefix) >> (shift + 8)) == 0;
                    ok = key != 0 && match;
                    d = (unsigned)(key >> shift) & 255u;
                }
                hist_add(wh, d, ok);
            }
            cluster_hist_total(cluster, S, buf);
            buf ^= 1;
            if (shift == NB - 8) {
                unsigned long long tot = 0;
                for (int b = 0; b < 256; ++b) tot += S.hsum[b];
                if (tot <= need) { all = true; break; }
            }
            scan_bins(S, need, true);
            const unsigned long long bin = S.bcast[0];
            const unsigned long long before = S.bcast[1];
            last_bin_count = S.hsum[bin];
            need -= before;
            prefix |= (K)bin << shift;
            __syncthreads();
        }
        if (!all) {
            tau = prefix;
            if (need < last_bin_count) {
                // more entries equal tau than may be kept: keep the `need`
                // smallest indices among them
                uint32_t ipre = 0;
                for (int shift = 24; shift >= 0; shift -= 8) {
                    for (int64_t e0 = 0; e0 < trip; e0 += blockDim.x) {
                        const int64_t e = e0 + tid;
                        bool ok = false;
                        unsigned d = 0;
                        if (e < nloc && Bits<T>::of(value(e)) == tau) {
                            const uint32_t ix = tie_index(e);
                            ok = shift == 24 ? true : ((ix ^ ipre) >> (shift + 8)) == 0;
                            d = (ix >> shift) & 255u;
                        }
                        hist_add(wh, d, ok);
                    }
                    cluster_hist_total(cluster, S, buf);
                    buf ^= 1;
                    scan_bins(S, need, false);
                    const unsigned long long bin = S.bcast[0];
                    need -= S.bcast[1];
                    ipre |= (uint32_t)bin << shift;
                    __syncthreads();
                }
                cut = ipre;
            }
        }
    }
    // the last totals read other CTAs' shared memory: no CTA may leave
    // before every CTA is done with them
    cluster.sync();
    if (keep_none) return;

    for (int64_t e = tid; e < nloc; e += blockDim.x) {
        const T x = value(e);
        const K key = Bits<T>::of(x);
        if (key == 0) continue;
        if (key < tau) continue;
        if (key == tau && tau != 0 && tie_index(e) > cut) continue;
        const int64_t g = lo + e;
        const int64_t c = matrix ? g / rows : (int64_t)seg;
        const int64_t i = matrix ? g - c * rows : g;
        const int pos = atomicAdd(&cnt[i], 1);
        if (pos >= k) {
            atomicOr(status, ST_OVERFLOW);
            continue;
        }
        colo[i * ld + pos] = (int32_t)c;
        valo[i * ld + pos] = x;
    }
}

template <typename T>
cudaError_t launch_select(const T* Xt, int64_t ldx, int64_t rows, int k,
                          int64_t t, int mode, EllDev out, unsigned* status,
                          cudaStream_t st, int sm_count, int64_t* smem_need_out)
{
    if (rows == 0) return cudaSuccess;
    const int nseg = mode == TOPT_MATRIX ? 1 : k;
    int C = sm_count / nseg;
    if (C > 8) C = 8;
    if (C < 1) C = 1;
    const int64_t seg_len = mode == TOPT_MATRIX ? (int64_t)k * rows : rows;
    int64_t per = (seg_len + C - 1) / C;
    per = (per + 3) & ~(int64_t)3;
    int64_t cache_elems = (int64_t)((kSelSmemMax - kSelFixedSmem) / sizeof(T));
    size_t smem = kSelFixedSmem;
    if (per <= cache_elems) {
        smem += (size_t)per * sizeof(T);
        cache_elems = per;
    } else {
        cache_elems = 0;
    }
    if (smem_need_out) *smem_need_out = (int64_t)smem;
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
    return cudaLaunchKernelEx(&cfg, select_kernel<T>, Xt, ldx, rows, k, t, mode,
                              out.cnt, out.col, static_cast<T*>(out.val),
                              cache_elems, status, out.ld);
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

template cudaError_t launch_select<float>(const float*, int64_t, int64_t, int, int64_t, int, EllDev, unsigned*, cudaStream_t, int, int64_t*);
template cudaError_t launch_select<double>(const double*, int64_t, int64_t, int, int64_t, int, EllDev, unsigned*, cudaStream_t, int, int64_t*);

}  // namespace espnmf
