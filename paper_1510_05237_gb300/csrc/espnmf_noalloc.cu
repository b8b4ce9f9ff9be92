// espnmf_noalloc.cu -- the stand-alone selector without any allocation.
//
// espnmf_enforce_topt_buffer takes its scratch memory (a column-major copy
// of X and the per-column thresholds) from the stream-ordered allocator on
// every call.  Some callers must not allocate device memory on their call
// path -- a service whose device memory is budgeted once at start-up, or a
// host that hands all device memory to its own pool -- so this variant runs
// the same kernels on a fixed scratch array that lives in this file:
//
//   static __device__ g_noalloc_scratch[kNoallocBytes]
//
// Every GPU that loads the library holds the array until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in), so every call, with the call's device current, asks
// the runtime for the array's device address (cudaGetSymbolAddress, which
// allocates nothing) rather than keeping an address that a device reset
// would make stale.  The first call on a device may load the library's
// device code there, so it should come before any stream capture.  All
// calls share the array and it keeps the previous call's contents: the
// parts that must start at zero are cleared on every call, and calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race on it.
#include <mutex>

#include "../../include/espnmf.h"
#include "common.cuh"

using namespace espnmf;

namespace {

// Largest rows * factor_ld(k) (and largest rows) one call may use.
constexpr int64_t kNoallocMaxElems = ESPNMF_NOALLOC_MAX_ELEMS;

constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
// Worst case over k <= 128 and element size 8: the column-major copy
// (k * ceil32(rows) <= MaxElems + 31 * 128 elements), the thresholds and
// tie cut-offs of up to 128 columns, and the status word.
constexpr size_t kXtBytes = a256((size_t)(kNoallocMaxElems + 31 * 128) * 8);
constexpr size_t kTauBytes = a256(128 * 8);
constexpr size_t kCutBytes = a256(128 * 4);
constexpr size_t kNoallocBytes = kXtBytes + kTauBytes + kCutBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_setup_mu;

// Failures are described through espnmf_last_error(NULL), like the other
// context-free calls.
espnmf_status fail(espnmf_status s, const char* msg, cudaError_t e = cudaSuccess)
{
    std::string m = msg;
    if (e != cudaSuccess) {
        m += ": ";
        m += cudaGetErrorString(e);
        cudaGetLastError();
    }
    set_thread_error(m.c_str());
    return s;
}

// Device address of the scratch array on the current device, looked up on
// every call, and the selector's kernel attributes set for that device.
espnmf_status scratch_for(unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(ESPNMF_ERR_CUDA, "cudaGetSymbolAddress", e);
    e = setup_select();
    if (e != cudaSuccess) return fail(ESPNMF_ERR_CUDA, "selector set-up", e);
    *out = static_cast<unsigned char*>(ptr);
    return ESPNMF_OK;
}

}  // namespace

extern "C" {

espnmf_status espnmf_enforce_topt_buffer_noalloc(void* X, int64_t rows, int32_t k, int64_t ld,
                                                 espnmf_dtype dtype, int64_t t,
                                                 espnmf_topt_mode mode, void* stream)
{
    set_thread_error("");
    if (!X || rows < 0 || k < 1 || k > 128 || ld < k || t < 0)
        return fail(ESPNMF_ERR_INVALID_ARG, "bad X/rows/k/ld/t");
    if (dtype != ESPNMF_F64 && dtype != ESPNMF_F32)
        return fail(ESPNMF_ERR_INVALID_ARG, "dtype must be F64 or F32");
    if (mode != ESPNMF_TOPT_COLUMN && mode != ESPNMF_TOPT_MATRIX && mode != ESPNMF_TOPT_NONE)
        return fail(ESPNMF_ERR_INVALID_ARG, "unknown enforcement mode");
    if (rows > kNoallocMaxElems || rows * (int64_t)factor_ld(k) > kNoallocMaxElems)
        return fail(ESPNMF_ERR_INVALID_ARG,
                    "X is larger than the static scratch allows (rows * ld(k) must be <= "
                    "ESPNMF_NOALLOC_MAX_ELEMS)");
    if (rows == 0) return ESPNMF_OK;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(ESPNMF_ERR_CUDA, "device", e);
    unsigned char* ws = nullptr;
    espnmf_status st0 = scratch_for(&ws);
    if (st0 != ESPNMF_OK) return st0;

    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = dtype == ESPNMF_F64 ? 8 : 4;
    const int64_t ldx = (rows + 31) / 32 * 32;
    const size_t bx = a256((size_t)k * ldx * es);
    if (bx + kTauBytes + kCutBytes + 256 > kNoallocBytes)
        return fail(ESPNMF_ERR_INVALID_ARG, "X is larger than the static scratch allows");
    void* tau = ws + bx;
    uint32_t* cut = (uint32_t*)(ws + bx + kTauBytes);
    unsigned* status = (unsigned*)(ws + bx + kTauBytes + kCutBytes);
    // the array keeps the last call's contents: clear the status word (the
    // rest is fully rewritten before it is read)
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = dtype == ESPNMF_F64
                ? launch_dense_to_colmajor<double, double>((const double*)X, rows, k, ld, (double*)ws, ldx, status, false, st)
                : launch_dense_to_colmajor<float, float>((const float*)X, rows, k, ld, (float*)ws, ldx, status, false, st);
    if (e == cudaSuccess)
        e = dtype == ESPNMF_F64
                ? launch_select<double>((const double*)ws, ldx, rows, k, t, (int)mode, tau, cut, st, sms, nullptr, nullptr)
                : launch_select<float>((const float*)ws, ldx, rows, k, t, (int)mode, tau, cut, st, sms, nullptr, nullptr);
    if (e == cudaSuccess)
        e = dtype == ESPNMF_F64 ? launch_apply_thresholds<double>((double*)X, rows, k, ld, (int)mode, tau, cut, status, st)
                                : launch_apply_thresholds<float>((float*)X, rows, k, ld, (int)mode, tau, cut, status, st);
    unsigned hstat = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ESPNMF_ERR_CUDA, "enforce_topt_buffer_noalloc", e);
    if (hstat & ST_NONFINITE) return fail(ESPNMF_ERR_NONFINITE, "non-finite value in X (X unchanged)");
    return ESPNMF_OK;
}

}  // extern "C"
