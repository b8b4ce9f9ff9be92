// common.cuh -- internal definitions shared by the library's translation
// units: device status flags, the on-device layouts of A and of the factors,
// and the launchers each kernel file exports.  Not part of the public ABI
// (that is include/espnmf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace espnmf {

// Bits of the device status word every kernel may raise (atomicOr).
enum : unsigned {
    ST_NONFINITE = 1u,   // a NaN/Inf met in an iterate
    ST_SINGULAR = 2u,    // Gram pivot (LDL^T d_j) below the singularity threshold
    ST_TIMEOUT = 4u,     // a bounded wait gave up
    ST_BADINPUT = 8u,    // negative entry in a factor given by the caller
    ST_OVERFLOW = 16u,   // a factor row received more than k entries (internal)
};

enum TopMode : int { TOPT_COLUMN = 0, TOPT_MATRIX = 1, TOPT_NONE = 2 };

// Checked build (compiled with -DESPNMF_CHECKED): bounds checks of the
// indexed accesses whose index comes from data -- a factor row gathered by
// the sparse product, a pair's column and a row's pair count, a frequent
// table slot, an output or partial row, a candidate or survivor row.  A
// failed check sets its bit in this translation unit's flag word and the
// access is skipped; espnmf_checked_flags() reports (and clears) the union
// over all kernels.  Without the flag ESPNMF_CHECK is the constant true and
// the checks compile to nothing.
enum : unsigned {
    CHK_FACTOR_ROW = 1u,   // gathered factor row >= the factor's rows
    CHK_COLUMN = 2u,       // a pair's column >= the row width
    CHK_COUNT = 4u,        // a row's pair count > its capacity
    CHK_SLOT = 8u,         // a frequent-table slot >= the table's rows
    CHK_OUT_ROW = 16u,     // an output or partial row out of range
    CHK_CAND_ROW = 32u,    // a candidate or survivor row >= the column length
};
#ifdef ESPNMF_CHECKED
static __device__ unsigned g_check_flags;
__device__ __forceinline__ bool espnmf_check(bool ok, unsigned bit)
{
    if (!ok) atomicOr(&g_check_flags, bit);
    return ok;
}
#define ESPNMF_CHECK(cond, bit) ::espnmf::espnmf_check((cond), (bit))
// Defines `unsigned name()` reading and clearing this unit's flag word.
#define ESPNMF_CHECK_READER(name)                                          \
    unsigned name()                                                        \
    {                                                                      \
        unsigned v = 0, z = 0;                                             \
        if (cudaMemcpyFromSymbol(&v, g_check_flags, sizeof v) != cudaSuccess) \
            return 0xffffffffu;                                            \
        cudaMemcpyToSymbol(g_check_flags, &z, sizeof z);                   \
        return v;                                                          \
    }
#else
#define ESPNMF_CHECK(cond, bit) true
#define ESPNMF_CHECK_READER(name) \
    unsigned name() { return 0; }
#endif
// y[0, count) = the FP32 values of the BF16 words x[0, count) (exact).
cudaError_t launch_bf16_to_f32(const uint16_t* x, int64_t count, float* y, cudaStream_t st);

// per translation unit: the flags its kernels raised (checked build)
unsigned check_flags_spmm();
unsigned check_flags_select();
unsigned check_flags_factor();
unsigned check_flags_seq();

// For non-negative IEEE numbers the bit pattern read as an unsigned integer
// orders exactly like the value; the selector works on these keys.
template <typename T> struct KeyBits;
template <> struct KeyBits<float> {
    using K = uint32_t;
    static constexpr int top_shift = 20;   // first histogram: bits 30..20
    __device__ static K of(float x) { return __float_as_uint(x); }
    __device__ static float value(K k) { return __uint_as_float(k); }
};
template <> struct KeyBits<double> {
    using K = unsigned long long;
    static constexpr int top_shift = 52;   // first histogram: the exponent
    __device__ static K of(double x) { return (K)__double_as_longlong(x); }
    __device__ static double value(K k) { return __longlong_as_double((long long)k); }
};

// Survival rule of the enforcement step, given the selector's threshold
// (tau, cut) for the entry's segment and the entry's tie index.
template <typename T>
__device__ __forceinline__ bool keep_entry(T v, typename KeyBits<T>::K tau, uint32_t cut,
                                           uint32_t ix)
{
    const typename KeyBits<T>::K key = KeyBits<T>::of(v);
    return key != 0 && (key > tau || (key == tau && ix <= cut));
}

// ---------------------------------------------------------------------------
// Compensated FP32 accumulation ("double-float": an unevaluated sum hi + lo
// of two floats).  The product of two floats is split exactly into p + e
// with one FMA (e = fma(a, b, -p)), and sums use Knuth's branch-free
// two-sum, so a running sum of products keeps about 48 significant bits --
// FP64-like accuracy -- on the FP32 pipes.  Used for per-lane sums in
// divergent code, where every FP64 warp instruction would hold the GPU's
// low-rate FP64 pipe whatever its active lanes; the sums are widened to
// FP64 (hi + lo) before they are reduced.
struct DFloat {
    float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void df_add(DFloat& s, float p, float e)
{
    const float t = s.hi + p;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (p - bp);
    const float lo = s.lo + (err + e);
    const float h = t + lo;
    s.lo = lo - (h - t);
    s.hi = h;
}
// s += a * b, the product exactly
__device__ __forceinline__ void df_add_prod(DFloat& s, float a, float b)
{
    const float p = __fmul_rn(a, b);   // never contracted into a neighbouring add
    df_add(s, p, fmaf(a, b, -p));
}
// s += (a - b)^2 with a - b split exactly (two-sum) first
__device__ __forceinline__ void df_add_sqdiff(DFloat& s, float a, float b)
{
    const float d = a - b;
    const float bb = d - a;
    const float dl = (a - (d - bb)) + (-b - bb);   // a - b = d + dl exactly
    const float p = __fmul_rn(d, d);
    df_add(s, p, fmaf(d, d, -p) + 2.f * d * dl);
}
__device__ __forceinline__ double df_value(const DFloat& s) { return (double)s.hi + (double)s.lo; }
// sum over the warp (every lane gets it), butterfly in a fixed order
__device__ __forceinline__ DFloat df_warp_sum(DFloat v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, v.hi, off);
        const float l = __shfl_xor_sync(0xffffffffu, v.lo, off);
        df_add(v, h, l);
    }
    return v;
}

// Rows are cut into segments of at most this many entries, one per lane.
constexpr int kSegTarget = 64;
constexpr int kMaxK = 256;

// ---------------------------------------------------------------------------
// A in sliced ELLPACK (SELL-32).  One layout per orientation: rows of A
// (n rows, gathers rows of V) and rows of A^T (m rows, gathers rows of U).
// A row is split into 1..32 segments of at most kSegTarget entries placed
// in adjacent lanes [head, end) of one slice (seg_grp = head << 8 | end);
// the lanes' sums are combined inside the warp.  Rows too long for 32
// segments are cut into chunks that write partial rows (seg_part >= 0),
// added by spmm_combine.  Lane l = s%32 of slice s/32 owns segment s; its
// entry p is at slice_ptr[s/32] + (p/4)*128 + 4*l + p%4 (slice lengths are
// multiples of 4), so a lane reads four entries with one 16-byte load and a
// warp 512 consecutive bytes.  Padding entries have idx = -1.
// One tier of a product's frequent part.  Each output row with entries in
// the tier holds them contiguously in ent[], padded with entries on the zero
// table row (value +0) to a multiple of `pad` (4 or the kernel's step, a
// divisor of 32); an entry is (byte offset of its table row, FP32 value
// bits).  rows[j] = (output row, end of its entries in units of four), the
// rows with entries in ascending order; chunk[c] .. chunk[c + 1] are the rows
// of work chunk c (about equal cost), which the warps of spmm_freq take in
// turn through `counter`.
struct FreqTierDev {
    int64_t nnz = 0;               // entries of A in the tier
    int64_t nent = 0;              // entries stored (padding included)
    uint2* ent = nullptr;          // [nent]
    int2* rows = nullptr;          // [nrows]
    int nrows = 0;
    int32_t* chunk = nullptr;      // [nchunks + 1]
    int nchunks = 0;
    int* counter = nullptr;        // next chunk to take (reset before each launch)
};

struct SellDev {
    int64_t rows = 0;        // output rows
    int64_t nseg = 0;
    int64_t nslices = 0;
    int64_t total = 0;       // stored entries, padding included
    int64_t nnz = 0;
    int64_t* slice_ptr = nullptr;  // [nslices+1]
    int32_t* slice_len = nullptr;  // [nslices]
    int32_t* idx = nullptr;        // [total]
    void* val = nullptr;           // [total] of T
    int32_t* seg_row = nullptr;    // [nslices*32], -1 for padding lanes
    int32_t* seg_part = nullptr;   // [nslices*32], partial slot or -1
    int32_t* seg_grp = nullptr;    // [nslices*32], head lane << 8 | end lane
    int64_t nsplit = 0;            // rows cut into segments
    int32_t* split_row = nullptr;  // [nsplit]
    int32_t* split_first = nullptr;// [nsplit] first partial slot
    int32_t* split_count = nullptr;// [nsplit]
    int64_t npart = 0;             // partial slots
    void* partials = nullptr;      // [npart * k] of T
    // Frequent part (FP32 form only; h = 0: none).  The h gathered rows that
    // the most entries reference (the frequent terms of A^T U) form a dense
    // table; their entries are kept out of the SELL arrays above and stored
    // per output row instead, in two tiers by the gathered row's slot:
    // tier 0 (slots < h1) is read by spmm_freq from the table staged in
    // shared memory, tier 1 (slots h1 .. h - 1) from the factor's table in
    // global memory.  slot_of[g] is the slot of gathered row g or -1.
    int h = 0;                     // table rows in all (slots 0 .. h - 1)
    int h1 = 0;                    // of them staged in shared memory (slots < h1)
    int32_t* slot_of = nullptr;    // [rows of the gathered factor]
    FreqTierDev ft[2];
};

// A factor (U: n x k, V: m x k) in row-packed sparse form: row i holds
// cnt[i] pairs (col[i*ld+q], val[i*ld+q]), q < cnt[i], columns distinct, all
// values > 0, pair order unspecified.  ld = factor_ld(k) keeps every row
// 16-byte aligned so a row's pairs load as 128-bit vectors.  Rows with at
// least `heavy` nonzeros also have a dense copy dense[i*ld + c] (zeros and
// the padding columns included), which the sparse product reads instead of
// the pairs.
//
// FP32 factors also keep, rewritten by every emit: a bitmask of the rows
// that hold a nonzero (bit r % 32 of word r / 32), and, when the sparse
// product that gathers this factor has a frequent part, the dense copy of
// each frequent row (htab[slot * ld + c], zeros and padding included) with
// a flag per slot telling whether the row is nonzero.
struct EllDev {
    int32_t* cnt = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;
    void* dense = nullptr;   // dense copies of heavy rows, row stride dld
    uint4* rec = nullptr;    // FP32 factors: per-row record (2 x uint4), see record_cnt
    int64_t rows = 0;        // rows of the factor
    uint32_t* nzmask = nullptr;      // FP32 factors: nonzero-row bitmask
    const int32_t* hslot = nullptr;  // [rows] slot in htab or -1 (nullptr: no table)
    void* htab = nullptr;            // [h][ld]
    uint8_t* hnz = nullptr;          // [h]
    int h = 0;
    int ld = 0;
    int dld = 0;
    int heavy = 1 << 30;
};

// Per-row record of an FP32 factor: 32 bytes (one L2 sector) in two 16-byte
// halves.  rec[2 i] = {cnt | c0 << 8 | c1 << 16 | c2 << 24, v0, v1, v2} and
// rec[2 i + 1] = {c3 | c4 << 8 | c5 << 16, v3, v4, v5}: the row's first six
// pairs in column order (c0 < c1 < ...), unused slots column 0 and value
// +0.  A row of up to three nonzeros is complete in the first half, one of
// up to six in the record.
__host__ __device__ inline int record_cnt(unsigned x) { return (int)(x & 0xffu); }

// Row stride of the dense heavy-row copies: 32 or 64 floats (whole 128-byte
// lines) up to k = 64, else the factor stride.
inline __host__ __device__ int dense_ld(int ld) { return ld <= 32 ? 32 : (ld <= 64 ? 64 : ld); }

// Row stride of factors, Y and the dense heavy rows: k rounded up to 4
// (k <= 64) or to 16.
inline __host__ __device__ int factor_ld(int k) { return k <= 64 ? (k + 3) / 4 * 4 : (k + 15) / 16 * 16; }
// A row with at least this many nonzeros is "heavy" (gathered densely).
inline __host__ __device__ int heavy_threshold(int ld) { return ld / 4 > 4 ? ld / 4 : 4; }

// ---------------------------------------------------------------------------
// Launchers.  Every launcher enqueues on `st` and returns the CUDA error of
// the launch.  T is float or double.

// Launch shape of the FP32 sparse product: the number of warps that share a
// slice's output columns (1, 2 or 4; k >= 13 for more than one), the
// preferred shared-memory carveout in percent (-1: the driver's choice) and
// whether zero factor rows are skipped by the bitmask.  Every shape computes
// bitwise the same Y.
struct SpmmConfig {
    int split = 1;
    int carveout = 100;   // the per-thread slots want all of the shared memory
    int mask = 1;   // skip zero factor rows by the bitmask: 0 no, 1 from global, 2 from shared
};
// Largest bitmask (32-bit words, i.e. factor rows / 32) that mask = 2 stages.
constexpr int kSellSmemMaskWords = 4096;

template <typename T>
cudaError_t launch_spmm(const SellDev& S, const EllDev& F, int k, T* Y,
                        int64_t ldy, SpmmConfig cfg, cudaStream_t st, int sm_count);
template <typename T>
cudaError_t launch_spmm_combine(const SellDev& S, int k, T* Y, int64_t ldy,
                                cudaStream_t st);
// Frequent part of an FP32 product (S.h > 0): Y += the products of the
// entries whose gathered row is one of the h frequent rows.  tier 1: the
// first S.h1 rows of F.htab staged in shared memory (TMA bulk copies;
// `wait_limit` bounds the wait for them); tier 2: the rows h1 .. h - 1 read
// from F.htab in global memory (L2).  Runs after launch_spmm (and the
// combine), tier 1 before tier 2, one CTA per SM.  Each warp streams its
// chunk's entries through a ring of kFreqStages stages of 32 entries in
// shared memory (cp.async).
constexpr int kHThreads = 1024;
constexpr int kFreqStages = 3;
constexpr size_t kHTableBytes = 200 * 1024;    // largest dense table staged
// entries per row of a tier are padded to a multiple of this (the entries a
// warp of spmm_freq adds per step, at least four)
int freq_pad(int ld);
constexpr size_t kH2TableBytes = 16u << 20;    // largest table of both tiers
constexpr int kMinTier2Rows = 256;             // a smaller second tier is not built
cudaError_t launch_spmm_h(const SellDev& S, const EllDev& F, float* Y, int sm_count,
                          unsigned* status, long long wait_limit, cudaStream_t st, int tier);

template <typename T>
cudaError_t launch_solve(const T* Y, int64_t ldy, int64_t rows, int k,
                         const T* Ginv, T* Xt, int64_t ldx, unsigned* status,
                         cudaStream_t st, int sm_count);

// Threshold of the enforcement step per column (or one for the whole matrix)
// from the column-major projected candidate Xt (k columns of length rows,
// leading dimension ldx, entries >= +0): tau[s] (key) and cut[s] (tie index).
// With rowbits (COLUMN mode), the survivors are also marked, bit c % 32 of
// word rowbits[i * ceil(k/32) + c / 32] (the words must be zero), and the
// FP64 sum of squares of each column's survivors is written to
// diag_part[c * select_cluster(...) + r], r < select_cluster(...).  With a
// hint (marking only: k keys, 0 = none), each column starts its search from
// the hint's threshold and stores its new threshold there; the result does
// not depend on the hint.  With counts, each column adds 1 to counts[0]
// when the hint's window held its threshold, else to counts[1].
template <typename T>
cudaError_t launch_select(const T* Xt, int64_t ldx, int64_t rows, int k,
                          int64_t t, int mode, void* tau, uint32_t* cut,
                          cudaStream_t st, int sm_count, uint32_t* rowbits,
                          double* diag_part, void* hint = nullptr,
                          unsigned long long* counts = nullptr);
int select_cluster(int64_t rows, int k, int mode, int sm_count);

// Projects and enforces a caller's dense rows x k buffer in place.
template <typename T>
cudaError_t launch_apply_thresholds(T* X, int64_t rows, int k, int64_t ld, int mode,
                                    const void* tau, const uint32_t* cut,
                                    unsigned* status, cudaStream_t st);

// Row-wise pass after the selector: writes the new factor's rows in column
// order (and dense copies of heavy rows), zeroes the old buffer's counts,
// and leaves per-block FP64 partials of the Gram matrix (entry-major:
// gram_part[e * nblocks + b]) and of ||F_new - F_old||^2, ||F_new||^2,
// ||F_old||^2 and <F_new, Y> (scal_part[j * nblocks + b]).
template <typename T>
cudaError_t launch_emit(const T* Xt, int64_t ldx, int64_t rows, int k, int mode,
                        const void* tau, const uint32_t* cut, EllDev cur, EllDev old,
                        bool residual, const T* Y, int64_t ldy, double* gram_part,
                        double* scal_part, int nblocks, cudaStream_t st);

struct MetricsArgs {
    bool enabled = false;
    const double* G_other = nullptr;   // V^T V (k x k) when reducing U^T U
    const double* A2 = nullptr;        // ||A||^2
    double* out = nullptr;             // [0] R, [1] E, [2] f = ||A-UV^T||^2
    double* hist_R = nullptr;
    double* hist_E = nullptr;
    int* hist_counter = nullptr;
    int hist_cap = 0;
};

// Adds the Gram partials (upper triangle, entry-major: gram_part[e * nparts
// + b] for e = tri(c, d), c <= d), the scalar partials (scal_part[j *
// nscal_parts + b]) and, for diagonal entries, diag_parts per-column partials
// (diag_part[c * diag_parts + j], or NULL) in a fixed order; writes the
// symmetric G and, with m.enabled, R and E.  With `pairs` every partial is a
// compensated FP32 pair (float2 hi, lo) in its 8-byte slot.
cudaError_t launch_gram_reduce(const double* gram_part, const double* scal_part, int nparts,
                               int nscal_parts, int k, const double* diag_part, int diag_parts,
                               bool pairs, double* G, double* scal, unsigned* counter,
                               MetricsArgs m, cudaStream_t st);

// Survivor-driven emit (FP32, column mode): rowbits from launch_select's
// marking (cleared here); nblocks blocks write partial columns [0, nblocks)
// of gram_part (P columns in all: the off-diagonal products of the rows
// with two or more nonzeros outside the frequent table) and of scal_part
// (nblocks columns).
cudaError_t launch_emit_s(const float* Xt, int64_t ldx, int64_t rows, int k, uint32_t* rowbits,
                          EllDev cur, EllDev old, bool residual, const float* Y, int64_t ldy,
                          double* gram_part, double* scal_part, int nblocks, int P,
                          cudaStream_t st);
// Off-diagonal Gram products of the frequent rows (F.htab), partial columns
// [pcol0, pcol0 + nblocks) of gram_part.
cudaError_t launch_gram_table(const EllDev& F, int k, double* gram_part, int P, int pcol0,
                              int nblocks, cudaStream_t st);

cudaError_t launch_error_metrics(const double* GU, const double* GV, int k,
                                 const double* A2, const double* cross,
                                 double* out, cudaStream_t st);

// Loss gradient and projected-gradient polish (k_grad.cu).
template <typename T, typename OutT>
cudaError_t launch_grad(int64_t rows, int k, const EllDev& F, const double* Go, const T* Y,
                        int64_t ldy, OutT* out, cudaStream_t st);
cudaError_t launch_lambda_max(const double* G, int k, double* eta_out, double* lam_out,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_pg_apply(int64_t rows, int k, const EllDev& F, const double* Go, const T* Y,
                            int64_t ldy, const double* eta, T* Xt, int64_t ldx, cudaStream_t st);

template <typename T>
cudaError_t launch_gram_inverse(const double* G, int k, double* Ginv64, T* GinvT,
                            unsigned* status, cudaStream_t st);

// FP32 form, KP = factor_ld(k) <= 64 (k_chol.cu): the FP64 Cholesky factor
// of G rounded to FP32 (strictly lower L and its transpose, KP x KP each,
// then the reciprocal diagonal, KP) and the row solves X = Y G^-1 by
// substitution, projected and written column-major.
cudaError_t launch_cholesky(const double* G, int k, int KP, float* Ls, float* LTs, float* rd,
                            unsigned* status, cudaStream_t st, float* Gh = nullptr,
                            float* Gl = nullptr);
// One step of iterative refinement (k_chol.cu): Xt holds x0 from
// launch_solve_chol with project = false; Gh, Gl the FP32 pair of G that
// launch_cholesky writes when given them.  Writes x0 + d projected into Xt,
// or (raw) unprojected row-major into out; with correct = false, d = 0
// (x0 only, e.g. to write it row-major).
cudaError_t launch_refine(const float* Y, int64_t ldy, const float* Yt, int64_t ldyt, int64_t rows,
                          int k, int KP, const float* L, const float* rd, const float* Gh,
                          const float* Gl, float* Xt, int64_t ldx, float* out, int64_t ldo,
                          bool raw, bool correct, unsigned* status, cudaStream_t st, int sm_count);
cudaError_t launch_solve_chol(const float* Y, int64_t ldy, int64_t rows, int k, int KP,
                              const float* L, const float* LT, const float* rd, float* Xt,
                              int64_t ldx, unsigned* status, cudaStream_t st, int sm_count,
                              bool project = true);
cudaError_t setup_chol();

// Alg. 3 (sequential ALS), a new block of k2 topics: g = G1^T F (k1 x k2)
// over the first k1 columns of G1 (rows_f x ld1, the fixed factor's
// converged topics) and the block factor F (row-packed: cnt, col, val with
// row stride ld), then Y[i][j] -= (H1 g)_ij for the rows_h rows of H1 (the
// updated factor's converged topics), j < k2.  k1 is read from device
// memory (*k1, at most k1_max), so a captured sweep serves every block; with
// k1 = 0 Y is left unchanged.  g holds k1_max * k2 doubles of scratch.
template <typename T>
cudaError_t launch_seq_deflate(int64_t rows_f, const T* G1, int64_t rows_h, const T* H1, int ld1,
                               int k1_max, const int* k1, int k2, const int32_t* cnt,
                               const int32_t* col, const T* val, int ld, double* g, T* Y,
                               int64_t ldy, cudaStream_t st);
// H[i * ld1 + j0 + j] = the block factor's value in row i, column j < k2.
template <typename T>
cudaError_t launch_seq_append(int64_t rows, const int32_t* cnt, const int32_t* col, const T* val,
                              int ld, int k2, T* H, int ld1, int j0, cudaStream_t st);

// out = sum of squares of val[0, count) and of the values of the entries
// ent2[0, count2) and ent3[0, count3) of the frequent tiers (NULL: none), in
// a fixed order.
template <typename T>
cudaError_t launch_norm2(const T* val, int64_t count, const uint2* ent2, int64_t count2,
                         const uint2* ent3, int64_t count3, double* part, int nparts,
                         double* out, cudaStream_t st);

// E for arbitrary U, V: cross term <U, Y> with Y = A V given.
template <typename T>
cudaError_t launch_ell_dot(int64_t rows, int k, EllDev F, const T* Y,
                           int64_t ldy, double* part, int nparts, double* out,
                           cudaStream_t st);

template <typename T>
cudaError_t launch_ell_to_colmajor(int64_t rows, int k, EllDev F, T* Xt,
                                   int64_t ldx, cudaStream_t st);

// Projected, column-major copy of a dense rows x k matrix (leading
// dimension ld); a non-finite entry raises ST_NONFINITE and, when
// reject_negative, a negative one ST_BADINPUT.
template <typename Tin, typename T>
cudaError_t launch_dense_to_colmajor(const Tin* X, int64_t rows, int k,
                                     int64_t ld, T* Xt, int64_t ldx,
                                     unsigned* status, bool reject_negative,
                                     cudaStream_t st);
template <typename T>
cudaError_t launch_ell_to_dense(int64_t rows, int k, EllDev F, T* X,
                                int64_t ld, cudaStream_t st);

// Document-clustering accuracy of each column of factor F (k_metrics.cu):
// hist (k x n_classes counters) is scratch; acc receives k doubles.  A
// label outside [0, n_classes) of a member row raises ST_BADINPUT.
cudaError_t launch_topic_accuracy(const EllDev& F, int k, const int32_t* labels, int n_classes,
                                  unsigned* hist, double* acc, unsigned* status, int sm_count,
                                  cudaStream_t st);

// Per-device one-time kernel attribute set-up (dynamic shared memory
// limits), called by espnmf_init before any launch or capture.
cudaError_t setup_spmm();
cudaError_t setup_solve();
cudaError_t setup_select();
cudaError_t setup_factor();

// Records the message espnmf_last_error(NULL) returns on this thread.
void set_thread_error(const char* msg);

// Kernel kinds the profiler keeps statistics for.
enum KernelKind : int {
    K_SPMM = 0, K_SPMM_T, K_COMBINE, K_SOLVE, K_SELECT, K_EMIT, K_GRAM_REDUCE,
    K_INVERSE, K_TO_COLMAJOR, K_NORM2, K_DOT, K_SCATTER, K_GRAD, K_LAMBDA, K_PG,
    K_SPMM_H, K_SPMM_H_T, K_GRAM_TABLE, K_REFINE, K_SPMM_H2, K_SPMM_H2_T, K_COUNT
};
const char* kernel_name(int kind);

}  // namespace espnmf
