// k_chol.cu -- the k x k solve of Alg. 2 steps 1 and 3 in the FP32 form
// (k <= 64), by a Cholesky factor instead of an explicit inverse:
//
//   cholesky      G = L L^T of the other factor's Gram matrix, in FP64, one
//                 CTA (right-looking, k^3 / 6 fused multiply-adds: a third
//                 of what an explicit inverse costs, which matters because
//                 FP64 runs at a small fraction of the FP32 rate on this
//                 GPU).  It writes L rounded to FP32: the strictly lower part
//                 row-major (Ls), its transpose (LTs) and the reciprocal
//                 diagonal (rd), each padded with zeros to KP columns.
//   solve_chol    per row y of Y: L z = y (forward), L^T x = z (backward),
//                 in FP32, one thread per row with the row in registers; the
//                 factor is read from shared memory with 128-bit broadcast
//                 loads.  The projection onto x >= 0 is fused and the result
//                 written column-major (Xt[c * ldx + row], coalesced across
//                 the threads of a warp) for the selector.
//
// An index j with G_jj = 0 belongs to an all-zero factor column: its row and
// column of L are zero and rd_j = 0, so x_j = 0 and no other entry depends on
// it (the minimum-norm solution).  Any other pivot (the j-th Schur
// complement diagonal, the same quantity the sweep-operator inverse tests)
// at or below 64 eps max_j G_jj raises ST_SINGULAR; a non-finite entry of G
// raises ST_NONFINITE.
#include <float.h>

#include "common.cuh"

namespace espnmf {

constexpr int kCholThreads = 256;

// 1 / sqrt(d) for d > 0: an FP32 seed r0 (relative error e0 < 2^-21) and
// one third-order step r = r0 (1 + e/2 + 3 e^2 / 8) with e = 1 - d r0^2
// (the Taylor series of (1 - e)^(-1/2)), which leaves an error of about
// e0^3 -- below FP64 rounding -- after five dependent FP64 operations.  The
// seed needs d and 1/sqrt(d) inside the normal FP32 range, so pivots outside
// [1e-30, 1e30] take the IEEE FP64 square root and division.
__device__ __forceinline__ double rsqrt_fp64(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    const double r0 = (double)rsqrtf((float)d);
    const double t = d * r0;
    const double e = fma(-t, r0, 1.0);
    const double q = e * fma(0.375, e, 0.5);
    return fma(r0, q, r0);
}

// Right-looking Cholesky on the lower triangle in shared memory, with
// look-ahead.  When step j starts, column j is already scaled (L_ij for
// i >= j).  Warp 0 then updates the next active column jn by column j,
// takes its pivot's reciprocal square root and scales it (the dependent
// FP64 chain of the factorisation), while the other warps update the rest
// of the trailing triangle (columns after jn, every lane on one entry of the
// packed suffix per pass); one barrier per step.  On this GPU every FP64
// warp instruction holds a sub-partition's FP64 pipe for many cycles, so the
// chain and the per-step barrier, not the k^3 / 6 multiply-adds, set the
// time (measured: 62 us for k = 50, against 71 us with two barriers a step
// and the chain after the update).
__global__ void __launch_bounds__(kCholThreads)
cholesky_kernel(const double* __restrict__ G, int k, int KP, float* __restrict__ Ls,
                float* __restrict__ LTs, float* __restrict__ rd, unsigned* status,
                float* __restrict__ Gh, float* __restrict__ Gl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ks = k + 1;                                   // row stride (odd)
    double* a = reinterpret_cast<double*>(smem_raw);        // [k][ks], lower part used
    int* act = reinterpret_cast<int*>(a + (size_t)k * ks);  // [k] 1: active index
    int* nxt = act + k;                                     // [k] next active index (k: none)
    // the lower triangle's entries (i, l) packed as i << 8 | l, ordered by
    // column l, then row i: the entries of columns > c are the suffix that
    // starts at cstart(c + 1)
    uint16_t* tri = reinterpret_cast<uint16_t*>(nxt + k);
    auto cstart = [&](int l) { return l * k - l * (l - 1) / 2; };
    __shared__ double tol;
    __shared__ int sing, nonfin, first;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e - i * k;
        if (j <= i) a[i * ks + j] = G[(size_t)i * k + j];
    }
    for (int l = tid; l < k; l += blockDim.x)
        for (int i = l; i < k; ++i) tri[cstart(l) + (i - l)] = (uint16_t)((i << 8) | l);
    if (tid == 0) {
        double md = 0.0;
        int nf = 0;
        for (int j = 0; j < k; ++j) {
            const double d = G[(size_t)j * k + j];
            if (!isfinite(d)) nf = 1;
            act[j] = (d != 0.0 && isfinite(d)) ? 1 : 0;
            if (act[j] && d > md) md = d;
        }
        int n = k;
        for (int j = k - 1; j >= 0; --j) {
            nxt[j] = n;
            if (act[j]) n = j;
        }
        first = n;
        tol = 64.0 * DBL_EPSILON * md;
        sing = 0;
        nonfin = nf;
    }
    __syncthreads();
    // warp 0: pivot and scale column c (whose entries are final)
    auto pivot_column = [&](int c) {
        const double d = a[c * ks + c];
        const bool bad = !(d > tol);
        const double r = rsqrt_fp64(bad ? 1.0 : d);
        if (bad && lane == 0) sing = 1;
        for (int i = c + 1 + lane; i < k; i += 32) a[i * ks + c] = act[i] ? a[i * ks + c] * r : 0.0;
        __syncwarp();
        if (lane == 0) a[c * ks + c] = r * d;   // L_cc = d / sqrt(d)
    };
    if (tid < 32 && first < k) pivot_column(first);
    __syncthreads();
    for (int j = first; j < k; j = nxt[j]) {
        const int jn = nxt[j];
        if (tid < 32) {
            if (jn < k) {
                // column jn by column j, then its pivot and scaling
                const double ljn = a[jn * ks + j];
                for (int i = jn + lane; i < k; i += 32)
                    a[i * ks + jn] = fma(-a[i * ks + j], ljn, a[i * ks + jn]);
                __syncwarp();
                pivot_column(jn);
            }
        } else if (jn + 1 < k) {
            // columns after jn: a_il -= L_ij L_lj (jn < l <= i)
            const int e0 = cstart(jn + 1), e1 = cstart(k);
            for (int e = e0 + tid - 32; e < e1; e += blockDim.x - 32) {
                const int il = tri[e];
                const int i = il >> 8, l = il & 0xff;
                a[i * ks + l] = fma(-a[i * ks + j], a[l * ks + j], a[i * ks + l]);
            }
        }
        __syncthreads();
    }
    // FP32 copies, zero-padded to KP x KP
    for (int e = tid; e < KP * KP; e += blockDim.x) {
        const int i = e / KP, l = e - i * KP;
        float v = 0.f;
        if (i < k && l < i && act[i] && act[l]) v = (float)a[i * ks + l];
        Ls[e] = v;                      // L[i][l], strictly lower
        LTs[(size_t)l * KP + i] = v;    // L^T[l][i]
    }
    for (int j = tid; j < KP; j += blockDim.x)
        rd[j] = (j < k && act[j]) ? (float)(1.0 / a[j * ks + j]) : 0.f;
    if (Gh) {
        // G itself as an unevaluated FP32 pair (hi + lo, about 48 bits), for
        // the residual of the refinement step
        for (int e = tid; e < KP * KP; e += blockDim.x) {
            const int i = e / KP, l = e - i * KP;
            const double g = (i < k && l < k) ? G[(size_t)i * k + l] : 0.0;
            const float h = (float)g;
            Gh[e] = h;
            Gl[e] = (float)(g - (double)h);
        }
    }
    if (tid == 0) {
        if (sing) atomicOr(status, ST_SINGULAR);
        if (nonfin) atomicOr(status, ST_NONFINITE);
    }
}

cudaError_t launch_cholesky(const double* G, int k, int KP, float* Ls, float* LTs, float* rd,
                            unsigned* status, cudaStream_t st, float* Gh, float* Gl)
{
    if (k < 1 || KP < k || KP > 64) return cudaErrorInvalidValue;
    const size_t smem = (size_t)k * (k + 1) * sizeof(double) + 2 * (size_t)k * sizeof(int) +
                        (size_t)k * (k + 1) / 2 * sizeof(uint16_t);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kCholThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;   // ahead of the concurrent SpMM's pending blocks
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cholesky_kernel, G, k, KP, Ls, LTs, rd, status, Gh, Gl);
}

// ---------------------------------------------------------------------------

constexpr int kSolveRows = 128;   // rows per tile, one per thread

// (s0, s1) = (a0 * b0 + s0, a1 * b1 + s1): one packed FP32 instruction, each
// lane rounded as fmaf rounds.
__device__ __forceinline__ void fma2f(float& s0, float& s1, float a0, float a1, float b0, float b1)
{
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(s0), "+f"(s1) : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// X = Y (F^T F)^-1 row by row, with F^T F = L L^T from cholesky_kernel, then
// the projection max(x, 0) (Alg. 2 steps 1 and 3).  Each thread solves R
// rows (rows r0 + tid and r0 + tid + kSolveRows), held in registers, so that
// every coefficient read from shared memory serves R rows.  Both
// substitutions run in column (axpy) form: once an unknown is final, it is
// multiplied into every unknown still open, so the updates of a step are
// independent of each other (two per packed FMA) instead of one dependent
// chain per unknown.  The negated factor is held in shared memory as
// N1[j][i] = -L[i][j] (i > j) and N2[j][i] = -L[j][i] (i < j), zero
// elsewhere, so a step reads its coefficients as aligned 16-byte rows; a
// zero coefficient leaves the unknown it meets unchanged.
template <int KP, int R>
__global__ void __launch_bounds__(kSolveRows, 4 / R)
solve_chol_kernel(const float* __restrict__ Y, int64_t ldy, int64_t rows, int k,
                  const float* __restrict__ Lg, const float* __restrict__ LTg,
                  const float* __restrict__ rdg, float* __restrict__ Xt, int64_t ldx,
                  unsigned* status, bool project)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* N1 = reinterpret_cast<float*>(smem_raw);   // [KP][KP]
    float* N2 = N1 + KP * KP;                           // [KP][KP]
    float* rds = N2 + KP * KP;                          // [KP]
    const int tid = threadIdx.x;
    for (int e = tid; e < KP * KP; e += blockDim.x) {
        const int j = e / KP, i = e - j * KP;
        const bool in = i < k && j < k;
        N1[e] = (in && i > j) ? -LTg[e] : 0.f;   // L^T[j][i] = L[i][j]
        N2[e] = (in && i < j) ? -Lg[e] : 0.f;    // L[j][i]
    }
    for (int e = tid; e < KP; e += blockDim.x) rds[e] = e < k ? rdg[e] : 0.f;
    __syncthreads();
    bool bad = false;
    for (int64_t r0 = (int64_t)blockIdx.x * kSolveRows * R; r0 < rows;
         r0 += (int64_t)gridDim.x * kSolveRows * R) {
        float x[R][KP];
#pragma unroll
        for (int h = 0; h < R; ++h) {
            const int64_t r = r0 + tid + h * kSolveRows;
            const bool live = r < rows;
            const float4* yr = reinterpret_cast<const float4*>(Y + (live ? r : 0) * ldy);
#pragma unroll
            for (int q = 0; q < KP / 4; ++q) {
                const float4 v = live ? yr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                x[h][4 * q + 0] = v.x;
                x[h][4 * q + 1] = v.y;
                x[h][4 * q + 2] = v.z;
                x[h][4 * q + 3] = v.w;
            }
        }
        // L z = y: z_j = x_j / L_jj, then x_i -= L_ij z_j for i > j
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            const float d = rds[j];
#pragma unroll
            for (int h = 0; h < R; ++h) x[h][j] *= d;
#pragma unroll
            for (int i = (j + 1) / 4 * 4; i < KP; i += 4) {
                const float4 l = *reinterpret_cast<const float4*>(N1 + j * KP + i);
#pragma unroll
                for (int h = 0; h < R; ++h) {
                    fma2f(x[h][i], x[h][i + 1], l.x, l.y, x[h][j], x[h][j]);
                    fma2f(x[h][i + 2], x[h][i + 3], l.z, l.w, x[h][j], x[h][j]);
                }
            }
        }
        // L^T x = z: x_j = z_j / L_jj, then z_i -= L_ji x_j for i < j
#pragma unroll
        for (int j = KP - 1; j >= 0; --j) {
            const float d = rds[j];
#pragma unroll
            for (int h = 0; h < R; ++h) x[h][j] *= d;
#pragma unroll
            for (int i = 0; i < (j + 3) / 4 * 4; i += 4) {
                const float4 l = *reinterpret_cast<const float4*>(N2 + j * KP + i);
#pragma unroll
                for (int h = 0; h < R; ++h) {
                    fma2f(x[h][i], x[h][i + 1], l.x, l.y, x[h][j], x[h][j]);
                    fma2f(x[h][i + 2], x[h][i + 3], l.z, l.w, x[h][j], x[h][j]);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < R; ++h) {
            const int64_t r = r0 + tid + h * kSolveRows;
            if (r < rows) {
#pragma unroll
                for (int c = 0; c < KP; ++c) {
                    if (c >= k) break;
                    const float v = x[h][c];
                    if (!isfinite(v)) bad = true;
                    Xt[(int64_t)c * ldx + r] = (v > 0.f || !project) ? v : 0.f;
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

// rows per thread of solve_chol_kernel.  Two rows per thread halve the
// shared-memory reads per FMA but need ~230 registers at k = 50 (8 warps per
// SM): measured slower on the 50k x 100k workload, so one.
constexpr int solve_rows_per_thread(int) { return 1; }

template <int KP>
static cudaError_t launch_solve_chol_kp(const float* Y, int64_t ldy, int64_t rows, int k,
                                        const float* L, const float* LT, const float* rd,
                                        float* Xt, int64_t ldx, unsigned* status,
                                        cudaStream_t st, int sm_count, bool project)
{
    const size_t smem = ((size_t)2 * KP * KP + KP) * sizeof(float);
    constexpr int R = solve_rows_per_thread(KP);
    const int64_t tiles = (rows + kSolveRows * R - 1) / (kSolveRows * R);
    int64_t grid = (int64_t)sm_count * (4 / R);
    if (grid > tiles) grid = tiles;
    solve_chol_kernel<KP, R><<<(unsigned)grid, kSolveRows, smem, st>>>(Y, ldy, rows, k, L, LT, rd,
                                                                     Xt, ldx, status, project);
    return cudaGetLastError();
}

cudaError_t launch_solve_chol(const float* Y, int64_t ldy, int64_t rows, int k, int KP,
                              const float* L, const float* LT, const float* rd, float* Xt,
                              int64_t ldx, unsigned* status, cudaStream_t st, int sm_count,
                              bool project)
{
    if (rows == 0) return cudaSuccess;
    if (ldy != KP) return cudaErrorInvalidValue;
    switch (KP) {
#define ESPNMF_KP(v) case v: return launch_solve_chol_kp<v>(Y, ldy, rows, k, L, LT, rd, Xt, ldx, status, st, sm_count, project);
        ESPNMF_KP(4) ESPNMF_KP(8) ESPNMF_KP(12) ESPNMF_KP(16) ESPNMF_KP(20) ESPNMF_KP(24)
        ESPNMF_KP(28) ESPNMF_KP(32) ESPNMF_KP(36) ESPNMF_KP(40) ESPNMF_KP(44) ESPNMF_KP(48)
        ESPNMF_KP(52) ESPNMF_KP(56) ESPNMF_KP(60) ESPNMF_KP(64)
#undef ESPNMF_KP
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// One step of iterative refinement of the solve.  solve_chol_kernel (run
// with project = false) leaves x0 = y (L L^T)^-1, unprojected, in Xt; this
// kernel forms the residual r = y - x0 G with G = Gh + Gl (an FP32 pair
// holding G to about 48 bits; each product split exactly by one FMA and
// the terms summed as a compensated pair), solves d = r (L L^T)^-1 by the
// same substitutions and writes x = x0 + d (projected into Xt, or raw and
// row-major).  The error of x0 is about cond(G) 2^-24 |x|, that of x about
// (cond(G) 2^-24)^2 |x| plus the final FP32 rounding: for cond(G) well
// below 2^12 the result is the FP64 solution rounded to FP32 within an ulp
// or two.  One thread per row; its x0 and r live in shared-memory columns
// and every loop runs at run time (an option, not the default path).
constexpr int kRefineRows = 128;

__global__ void __launch_bounds__(kRefineRows)
refine_kernel(const float* __restrict__ Y, int64_t ldy, const float* __restrict__ Yt,
              int64_t ldyt, int64_t rows, int k, int KP, const float* __restrict__ Lg,
              const float* __restrict__ LTg, const float* __restrict__ rdg,
              const float* __restrict__ Ghg, const float* __restrict__ Glg,
              float* __restrict__ Xt, int64_t ldx, float* __restrict__ out, int64_t ldo,
              bool raw, bool correct, unsigned* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int B = kRefineRows;
    float* L = reinterpret_cast<float*>(smem_raw);   // [KP][KP] L[i][l], strictly lower
    float* Gh = L + KP * KP;                           // [KP][KP]
    float* Gl = Gh + KP * KP;                          // [KP][KP]
    float* rds = Gl + KP * KP;                         // [KP]
    float* xs = rds + KP;                              // [KP][B] x0 by column
    float* ds = xs + KP * B;                           // [KP][B] r, then d
    const int tid = threadIdx.x;
    for (int e = tid; e < KP * KP; e += blockDim.x) {
        L[e] = Lg[e];
        Gh[e] = correct ? Ghg[e] : 0.f;
        Gl[e] = correct ? Glg[e] : 0.f;
    }
    for (int e = tid; e < KP; e += blockDim.x) rds[e] = e < k ? rdg[e] : 0.f;
    (void)LTg;
    __syncthreads();
    bool bad = false;
    float* x = xs + tid;
    float* d = ds + tid;
    for (int64_t r0 = (int64_t)blockIdx.x * B; r0 < rows; r0 += (int64_t)gridDim.x * B) {
        const int64_t r = r0 + tid;
        if (r >= rows) continue;   // no barrier below
        for (int c = 0; c < k; ++c) x[c * B] = Xt[(int64_t)c * ldx + r];
        for (int c = 0; c < k; ++c) d[c * B] = 0.f;
        // residual, compensated
        for (int j = 0; j < (correct ? k : 0); ++j) {
            DFloat s;
            s.hi = Y ? Y[r * ldy + j] : 0.f;
            if (Yt) df_add(s, Yt[(int64_t)j * ldyt + r], 0.f);
            float tail = 0.f;
            for (int l = 0; l < k; ++l) {
                const float xl = x[l * B];
                df_add_prod(s, -xl, Gh[l * KP + j]);
                tail = __fmaf_rn(-xl, Gl[l * KP + j], tail);
            }
            d[j * B] = s.hi + (s.lo + tail);
        }
        // d (L L^T)^-1: L z = d, then L^T x = z (inactive indices have rds 0)
        for (int j = 0; j < (correct ? k : 0); ++j) {
            float v = d[j * B];
            for (int l = 0; l < j; ++l) v = __fmaf_rn(-L[j * KP + l], d[l * B], v);
            d[j * B] = v * rds[j];
        }
        for (int j = correct ? k - 1 : -1; j >= 0; --j) {
            float v = d[j * B];
            for (int l = j + 1; l < k; ++l) v = __fmaf_rn(-L[l * KP + j], d[l * B], v);
            d[j * B] = v * rds[j];
        }
        for (int c = 0; c < k; ++c) {
            const float v = x[c * B] + d[c * B];
            if (!isfinite(v)) bad = true;
            if (raw) out[r * ldo + c] = v;
            else Xt[(int64_t)c * ldx + r] = v > 0.f ? v : 0.f;
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

static size_t refine_smem(int KP) { return ((size_t)3 * KP * KP + KP + (size_t)2 * KP * kRefineRows) * sizeof(float); }

cudaError_t launch_refine(const float* Y, int64_t ldy, const float* Yt, int64_t ldyt, int64_t rows,
                          int k, int KP, const float* L, const float* rd, const float* Gh,
                          const float* Gl, float* Xt, int64_t ldx, float* out, int64_t ldo,
                          bool raw, bool correct, unsigned* status, cudaStream_t st, int sm_count)
{
    if (rows == 0) return cudaSuccess;
    if ((correct && ((!Y && !Yt) || !Gh || !Gl)) || KP > 64 || k > KP) return cudaErrorInvalidValue;
    const int64_t tiles = (rows + kRefineRows - 1) / kRefineRows;
    int64_t grid = (int64_t)sm_count * 2;
    if (grid > tiles) grid = tiles;
    refine_kernel<<<(unsigned)grid, kRefineRows, refine_smem(KP), st>>>(
        Y, ldy, Yt, ldyt, rows, k, KP, L, nullptr, rd, Gh, Gl, Xt, ldx, out, ldo, raw, correct, status);
    return cudaGetLastError();
}

template <int KP>
static cudaError_t setup_solve_kp()
{
    const size_t smem = ((size_t)2 * KP * KP + KP) * sizeof(float);
    constexpr int R = solve_rows_per_thread(KP);
    cudaError_t e = cudaFuncSetAttribute(solve_chol_kernel<KP, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);

    // four blocks per SM need most of the shared memory: do not let the
    // driver pick a smaller carveout
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_chol_kernel<KP, R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t setup_chol()
{
    {
        cudaError_t e0 = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)refine_smem(64));
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         64 * 65 * 8 + 2 * 64 * 4 + 64 * 65);
#define ESPNMF_KP(v) if (e == cudaSuccess) e = setup_solve_kp<v>();
    ESPNMF_KP(4) ESPNMF_KP(8) ESPNMF_KP(12) ESPNMF_KP(16) ESPNMF_KP(20) ESPNMF_KP(24)
    ESPNMF_KP(28) ESPNMF_KP(32) ESPNMF_KP(36) ESPNMF_KP(40) ESPNMF_KP(44) ESPNMF_KP(48)
    ESPNMF_KP(52) ESPNMF_KP(56) ESPNMF_KP(60) ESPNMF_KP(64)
#undef ESPNMF_KP
    return e;
}

}  // namespace espnmf
