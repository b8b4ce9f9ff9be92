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
    ST_SINGULAR = 2u,    // Cholesky pivot below the singularity threshold
    ST_TIMEOUT = 4u,     // a bounded wait gave up
    ST_BADINPUT = 8u,    // negative entry in a factor given by the caller
    ST_OVERFLOW = 16u,   // a factor row received more than k entries (internal)
};

enum TopMode : int { TOPT_COLUMN = 0, TOPT_MATRIX = 1, TOPT_NONE = 2 };

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
// added by spmm_combine.  Lane s%32 of slice s/32 owns segment s; its entry
// p is at slice_ptr[s/32] + p*32 + s%32, so a warp reads 32 consecutive
// entries per step.  Padding entries have idx = -1.
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
};

// A factor (U: n x k, V: m x k) in row-packed sparse form: row i holds
// cnt[i] pairs (col[i*ld+q], val[i*ld+q]), q < cnt[i], columns distinct, all
// values > 0, pair order unspecified.  ld = factor_ld(k) keeps every row
// 16-byte aligned so a row's pairs load as 128-bit vectors.  Rows with at
// least `heavy` nonzeros also have a dense copy dense[i*ld + c] (zeros and
// the padding columns included), which the sparse product reads instead of
// the pairs.
struct EllDev {
    int32_t* cnt = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;
    void* dense = nullptr;
    int ld = 0;
    int heavy = 1 << 30;
};

// Row stride of factors, Y and the dense heavy rows: k rounded up to 4
// (k <= 64) or to 16.
inline __host__ __device__ int factor_ld(int k) { return k <= 64 ? (k + 3) / 4 * 4 : (k + 15) / 16 * 16; }
// A row with at least this many nonzeros is "heavy" (gathered densely).
inline __host__ __device__ int heavy_threshold(int ld) { return ld / 4 > 4 ? ld / 4 : 4; }

// ---------------------------------------------------------------------------
// Launchers.  Every launcher enqueues on `st` and returns the CUDA error of
// the launch.  T is float or double.

template <typename T>
cudaError_t launch_spmm(const SellDev& S, const EllDev& F, int k, T* Y,
                        int64_t ldy, cudaStream_t st, int sm_count);
template <typename T>
cudaError_t launch_spmm_combine(const SellDev& S, int k, T* Y, int64_t ldy,
                                cudaStream_t st);

template <typename T>
cudaError_t launch_solve(const T* Y, int64_t ldy, int64_t rows, int k,
                         const T* Ginv, T* Xt, int64_t ldx, unsigned* status,
                         cudaStream_t st, int sm_count);

// Top-t selection on the column-major candidate Xt (k columns of length
// rows, leading dimension ldx, entries >= +0, padding rows are +0), writing
// the kept entries into the row-packed factor `out` (out.cnt zeroed
// beforehand).
template <typename T>
cudaError_t launch_select(const T* Xt, int64_t ldx, int64_t rows, int k,
                          int64_t t, int mode, EllDev out, unsigned* status,
                          cudaStream_t st, int sm_count,
                          int64_t* smem_need_out = nullptr);

// Row-wise pass over a freshly written factor: per-block FP64 Gram
// partials, residual/error partials, and zeroing of the previous buffer's
// counts.
template <typename T>
cudaError_t launch_finalize(int64_t rows, int k, EllDev cur, EllDev old,
                            bool residual, bool zero_old, const T* Y,
                            int64_t ldy, double* gram_part,
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

cudaError_t launch_gram_reduce(const double* gram_part,
                               const double* scal_part, int nparts, int k,
                               double* G, double* scal, unsigned* counter,
                               MetricsArgs m, cudaStream_t st);

cudaError_t launch_error_metrics(const double* GU, const double* GV, int k,
                                 const double* A2, const double* cross,
                                 double* out, cudaStream_t st);

template <typename T>
cudaError_t launch_cholesky(const double* G, int k, double* Ginv64, T* GinvT,
                            unsigned* status, cudaStream_t st);

template <typename Tin, typename T>
cudaError_t launch_dense_to_ell(const Tin* F, int64_t rows, int k, EllDev out,
                                unsigned* status, cudaStream_t st);

template <typename T>
cudaError_t launch_norm2(const T* val, int64_t count, double* part,
                         int nparts, double* out, cudaStream_t st);

// E for arbitrary U, V: cross term <U, Y> with Y = A V given.
template <typename T>
cudaError_t launch_ell_dot(int64_t rows, int k, EllDev F, const T* Y,
                           int64_t ldy, double* part, int nparts, double* out,
                           cudaStream_t st);

template <typename T>
cudaError_t launch_ell_to_colmajor(int64_t rows, int k, EllDev F, T* Xt,
                                   int64_t ldx, cudaStream_t st);

template <typename T>
cudaError_t launch_dense_to_colmajor(const T* X, int64_t rows, int k,
                                     int64_t ld, T* Xt, int64_t ldx,
                                     unsigned* status, cudaStream_t st);
template <typename T>
cudaError_t launch_ell_to_dense(int64_t rows, int k, EllDev F, T* X,
                                int64_t ld, cudaStream_t st);

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
    K_SPMM = 0, K_COMBINE, K_SOLVE, K_SELECT, K_FINALIZE, K_GRAM_REDUCE,
    K_CHOLESKY, K_DENSE_TO_ELL, K_NORM2, K_DOT, K_SCATTER, K_COUNT
};
const char* kernel_name(int kind);

}  // namespace espnmf
