// k_factor.cu -- everything that happens to a factor after its selection:
//
//   finalize      row-wise pass over the new factor: per-block FP64 partial
//                 sums of its Gram matrix F^T F (the "U^T U" / "V^T V" of
//                 Alg. 2 steps 1 and 3), of ||F_new - F_old||^2, ||F_new||^2,
//                 ||F_old||^2 (Sec. 3.1 residual) and of <U, A V> (the cross
//                 term of the error identity); zeroes the old buffer's counts.
//   gram_reduce   adds the block partials in a fixed order; its last block
//                 also forms R and E (Sec. 3.1) without ever forming U V^T:
//                 E^2 ||A||^2 = ||A||^2 - 2 <U, A V> + <U^T U, V^T V>.
//   cholesky      FP64 Cholesky factorisation of the Gram matrix and its
//                 inverse (one CTA), used by the k x k solve.
//   conversions   dense -> row-packed, row-packed -> dense / column-major,
//                 ||A||^2 and the stand-alone <U, Y> reduction.
//
// Every reduction adds in a fixed order (per warp, then per block in warp
// order, then over blocks in block order), so all results are reproducible.
#include <float.h>

#include "common.cuh"

namespace espnmf {

static __host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
struct FinArgs {
    int64_t rows;
    int k;
    int ld;
    int heavy;
    const int32_t* cnt_new;
    const int32_t* col_new;
    const T* val_new;
    T* dense_new;          // dense copies of heavy rows (may be null)
    int32_t* cnt_old;
    const int32_t* col_old;
    const T* val_old;
    bool residual;
    bool zero_old;
    const T* Y;
    int64_t ldy;
    double* gram_part;
    double* scal_part;
};

template <typename T>
static __host__ __device__ size_t fin_warp_bytes(int k, int ld, bool residual)
{
    // Gram accumulator, staged rows (columns, values), and per-lane dense
    // scratch rows of the new (and old) values, slot c of lane l at c*32+l
    return align16((size_t)k * k * sizeof(double)) + align16((size_t)32 * ld * sizeof(int)) +
           align16((size_t)32 * ld * sizeof(T)) + align16((size_t)32 * k * sizeof(T)) +
           (residual ? align16((size_t)32 * k * sizeof(T)) : 0);
}

__device__ inline double warp_sum(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Copies n (a multiple of 4 not exceeding the row stride) ints / values of
// a 16-byte aligned row with 128-bit loads.
__device__ inline void copy_row4(int* dst, const int32_t* src, int n)
{
    for (int q = 0; q < n; q += 4) *reinterpret_cast<int4*>(dst + q) = __ldg(reinterpret_cast<const int4*>(src + q));
}
__device__ inline void copy_row4(float* dst, const float* src, int n)
{
    for (int q = 0; q < n; q += 4) *reinterpret_cast<float4*>(dst + q) = __ldg(reinterpret_cast<const float4*>(src + q));
}
__device__ inline void copy_row4(double* dst, const double* src, int n)
{
    for (int q = 0; q < n; q += 2) *reinterpret_cast<double2*>(dst + q) = __ldg(reinterpret_cast<const double2*>(src + q));
}

template <typename T>
__global__ void __launch_bounds__(128)
finalize_kernel(FinArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][4];
    const int k = a.k, ld = a.ld;
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t pw = fin_warp_bytes<T>(k, ld, a.residual);
    unsigned char* wbase = smem_raw + warp * pw;
    double* G = reinterpret_cast<double*>(wbase);
    int* sc = reinterpret_cast<int*>(wbase + align16((size_t)k * k * sizeof(double)));
    T* sv = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(sc) + align16((size_t)32 * ld * sizeof(int)));
    T* sn = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(sv) + align16((size_t)32 * ld * sizeof(T)));
    T* so = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(sn) + align16((size_t)32 * k * sizeof(T)));
    for (int e = lane; e < k * k; e += 32) G[e] = 0.0;
    for (int e = lane; e < 32 * k; e += 32) sn[e] = T(0);
    if (a.residual)
        for (int e = lane; e < 32 * k; e += 32) so[e] = T(0);
    double s_diff = 0.0, s_new = 0.0, s_old = 0.0, s_cross = 0.0;

    const int64_t chunk = (a.rows + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < a.rows ? b0 + chunk : a.rows;
    __syncwarp();
    for (int64_t base = b0 + (int64_t)warp * 32; base < b1; base += (int64_t)W * 32) {
        const int64_t r = base + lane;
        const bool valid = r < b1;
        const int Ln = valid ? a.cnt_new[r] : 0;
        const int Ln4 = (Ln + 3) & ~3;
        int* mc = sc + lane * ld;
        T* mv = sv + lane * ld;
        copy_row4(mc, a.col_new + r * ld, Ln4);
        copy_row4(mv, a.val_new + r * ld, Ln4);
        for (int q = 0; q < Ln; ++q) sn[mc[q] * 32 + lane] = mv[q];
        if (a.dense_new && Ln >= a.heavy) {
            T* dr = a.dense_new + r * ld;
            for (int c = 0; c < ld; ++c) dr[c] = c < k ? sn[c * 32 + lane] : T(0);
        }
        int Lo = 0;
        if (valid && (a.residual || a.zero_old)) {
            Lo = a.cnt_old[r];
            if (a.residual) {
                const int32_t* co = a.col_old + r * ld;
                const T* vo = a.val_old + r * ld;
                for (int q = 0; q < Lo; ++q) so[co[q] * 32 + lane] = vo[q];
            }
            if (a.zero_old) a.cnt_old[r] = 0;
        }
        // row sums in column order (independent of the pair order in a row)
        if (Ln > 0 || Lo > 0) {
            for (int c = 0; c < k; ++c) {
                const double n = (double)sn[c * 32 + lane];
                s_new += n * n;
                if (a.Y && n != 0.0) s_cross += n * (double)a.Y[r * a.ldy + c];
                if (a.residual) {
                    const double o = (double)so[c * 32 + lane];
                    s_old += o * o;
                    s_diff += (n - o) * (n - o);
                    so[c * 32 + lane] = T(0);
                }
                sn[c * 32 + lane] = T(0);
            }
        }
        __syncwarp();
        // Gram: the 32 staged rows one after another; a row's pairs (ia <= ib)
        // across the lanes, accumulated into the upper triangle (canonical
        // slot min(c,d)*k + max(c,d)); distinct slots within a row.
        for (int j = 0; j < 32; ++j) {
            const int Lj = __shfl_sync(0xffffffffu, Ln, j);
            const int* jc = sc + j * ld;
            const T* jv = sv + j * ld;
            for (int ia = 0; ia < Lj; ++ia) {
                const int ca = jc[ia];
                const double va = (double)jv[ia];
                for (int ib = ia + lane; ib < Lj; ib += 64) {
                    const int cb = jc[ib];
                    const int s0 = ca < cb ? ca * k + cb : cb * k + ca;
                    const double p0 = va * (double)jv[ib];
                    const int ib2 = ib + 32;
                    if (ib2 < Lj) {
                        const int cb2 = jc[ib2];
                        const int s1 = ca < cb2 ? ca * k + cb2 : cb2 * k + ca;
                        const double p1 = va * (double)jv[ib2];
                        G[s0] += p0;
                        G[s1] += p1;
                    } else {
                        G[s0] += p0;
                    }
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // block partial: warps in order, upper triangle mirrored
    double* gp = a.gram_part + (size_t)blockIdx.x * k * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int c = e / k, d = e - c * k;
        const int src = c <= d ? c * k + d : d * k + c;
        double sum = 0.0;
        for (int w = 0; w < W; ++w)
            sum += reinterpret_cast<const double*>(smem_raw + w * pw)[src];
        gp[e] = sum;
    }
    s_diff = warp_sum(s_diff);
    s_new = warp_sum(s_new);
    s_old = warp_sum(s_old);
    s_cross = warp_sum(s_cross);
    if (lane == 0) {
        red[warp][0] = s_diff;
        red[warp][1] = s_new;
        red[warp][2] = s_old;
        red[warp][3] = s_cross;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double sum = 0.0;
        for (int w = 0; w < W; ++w) sum += red[w][threadIdx.x];
        a.scal_part[(size_t)blockIdx.x * 4 + threadIdx.x] = sum;
    }
}

template <typename T>
cudaError_t launch_finalize(int64_t rows, int k, EllDev cur, EllDev old,
                            bool residual, bool zero_old, const T* Y,
                            int64_t ldy, double* gram_part,
                            double* scal_part, int nblocks, cudaStream_t st)
{
    FinArgs<T> a;
    a.rows = rows;
    a.k = k;
    a.ld = cur.ld;
    a.heavy = cur.heavy;
    a.cnt_new = cur.cnt;
    a.col_new = cur.col;
    a.val_new = static_cast<const T*>(cur.val);
    a.dense_new = static_cast<T*>(cur.dense);
    a.cnt_old = old.cnt;
    a.col_old = old.col;
    a.val_old = static_cast<const T*>(old.val);
    a.residual = residual && old.cnt != nullptr;
    a.zero_old = zero_old && old.cnt != nullptr;
    a.Y = Y;
    a.ldy = ldy;
    a.gram_part = gram_part;
    a.scal_part = scal_part;
    const size_t pw = fin_warp_bytes<T>(k, cur.ld, a.residual);
    int W = (int)((210 * 1024) / pw);
    if (W > 4) W = 4;
    if (W < 1) W = 1;
    finalize_kernel<T><<<nblocks, W * 32, W * pw, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

__global__ void gram_reduce_kernel(const double* __restrict__ gram_part,
                                   const double* __restrict__ scal_part,
                                   int P, int k, double* G, double* scal,
                                   unsigned* counter, MetricsArgs m)
{
    const int kk = k * k;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    // eight interleaved partial sums, combined in a fixed order (FP64 adds
    // have a long latency on this part)
    if (e < kk) {
        double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int p = 0;
        for (; p + 7 < P; p += 8)
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] += gram_part[(size_t)(p + u) * kk + e];
        for (; p < P; ++p) s[0] += gram_part[(size_t)p * kk + e];
        G[e] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int p = 0;
        for (; p + 7 < P; p += 8)
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] += scal_part[(size_t)(p + u) * 4 + threadIdx.x];
        for (; p < P; ++p) s[0] += scal_part[(size_t)p * 4 + threadIdx.x];
        scal[threadIdx.x] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
    }
    if (!m.enabled) return;
    // The last block to finish forms the measures.
    __shared__ bool last;
    __shared__ double red[32];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tr = 0.0;
    for (int q = threadIdx.x; q < kk; q += blockDim.x) tr += __ldcg(G + q) * m.G_other[q];
    tr = warp_sum(tr);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = tr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double diff = __ldcg(scal + 0), nw = __ldcg(scal + 1);
        const double od = __ldcg(scal + 2), cross = __ldcg(scal + 3);
        double R;
        if (nw == 0.0) R = od == 0.0 ? 0.0 : __longlong_as_double(0x7ff0000000000000ll);
        else R = sqrt(diff) / sqrt(nw);
        const double A2 = *m.A2;
        const double f = A2 - 2.0 * cross + t;
        const double E = A2 == 0.0 ? 0.0 : sqrt(f > 0.0 ? f : 0.0) / sqrt(A2);
        m.out[0] = R;
        m.out[1] = E;
        m.out[2] = f;
        m.out[3] = t;
        if (m.hist_counter) {
            const int slot = *m.hist_counter;
            if (slot < m.hist_cap) {
                m.hist_R[slot] = R;
                m.hist_E[slot] = E;
            }
            *m.hist_counter = slot + 1;
        }
        *counter = 0u;
    }
}

cudaError_t launch_gram_reduce(const double* gram_part,
                               const double* scal_part, int nparts, int k,
                               double* G, double* scal, unsigned* counter,
                               MetricsArgs m, cudaStream_t st)
{
    const int B = 256;
    const int grid = (k * k + B - 1) / B;
    gram_reduce_kernel<<<grid, B, 0, st>>>(gram_part, scal_part, nparts, k, G,
                                           scal, counter, m);
    return cudaGetLastError();
}

// E for the current U, V from ||A||^2, <U, A V> (already reduced into
// *cross) and <U^T U, V^T V>; writes out[1] = E, out[2] = f, out[3] = trace.
__global__ void error_metrics_kernel(const double* __restrict__ GU,
                                     const double* __restrict__ GV, int k,
                                     const double* A2, const double* cross,
                                     double* out)
{
    __shared__ double red[32];
    double tr = 0.0;
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) tr += GU[q] * GV[q];
    tr = warp_sum(tr);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double a2 = *A2;
        const double f = a2 - 2.0 * (*cross) + t;
        out[1] = a2 == 0.0 ? 0.0 : sqrt(f > 0.0 ? f : 0.0) / sqrt(a2);
        out[2] = f;
        out[3] = t;
    }
}

cudaError_t launch_error_metrics(const double* GU, const double* GV, int k,
                                 const double* A2, const double* cross,
                                 double* out, cudaStream_t st)
{
    error_metrics_kernel<<<1, 256, 0, st>>>(GU, GV, k, A2, cross, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 Cholesky G = L L^T and G^-1 = L^-T L^-1 in one CTA.  An index whose
// diagonal is exactly 0 belongs to an all-zero factor column: it is taken
// out (identity row/column during the factorisation, zero row/column in the
// inverse), which gives the minimum-norm solution.  A pivot <= 64 eps
// max_j G_jj elsewhere raises ST_SINGULAR.

template <typename T>
__global__ void __launch_bounds__(1024)
cholesky_kernel(const double* __restrict__ G, int k, double* Ginv64,
                T* GinvT, unsigned* status, int li_in_smem)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* A = reinterpret_cast<double*>(smem_raw);                 // k*k
    double* Li = li_in_smem ? A + (size_t)k * k : Ginv64;             // k*k
    double* dinv = A + (size_t)k * k * (li_in_smem ? 2 : 1);          // k
    int* act = reinterpret_cast<int*>(dinv + k);
    __shared__ double inv_piv, maxdiag;
    __shared__ int sing, nonfin;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int kk = k * k;
    for (int e = tid; e < kk; e += nt) A[e] = G[e];
    __syncthreads();
    if (tid == 0) {
        double md = 0.0;
        int nf = 0;
        for (int j = 0; j < k; ++j) {
            const double d = A[j * k + j];
            if (!isfinite(d)) nf = 1;
            act[j] = d != 0.0 && isfinite(d);
            if (act[j] && d > md) md = d;
        }
        maxdiag = md;
        sing = 0;
        nonfin = nf;
    }
    __syncthreads();
    for (int e = tid; e < kk; e += nt) {
        const int i = e / k, j = e - i * k;
        if (!act[i] || !act[j]) A[e] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    const double tol = 64.0 * DBL_EPSILON * maxdiag;
    // right-looking Cholesky, lower triangle of A
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            double s = A[j * k + j];
            if (act[j] && !(s > tol)) {
                sing = 1;
                s = 1.0;
            }
            const double ri = rsqrt(s);
            A[j * k + j] = s * ri;   // sqrt(s)
            inv_piv = ri;
            dinv[j] = ri;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < k; i += nt) A[i * k + j] *= inv_piv;
        __syncthreads();
        const int nrem = k - j - 1;
        for (int e = tid; e < nrem * nrem; e += nt) {
            const int ii = e / nrem, ll = e - ii * nrem;
            if (ll <= ii) {
                const int i = j + 1 + ii, l = j + 1 + ll;
                A[i * k + l] -= A[i * k + j] * A[l * k + j];
            }
        }
        __syncthreads();
    }
    // Li = L^-1 (lower), row by row; each entry a dot product split over
    // four independent accumulators (FP64 FMA latency is long on this part).
    for (int i = 0; i < k; ++i) {
        const double di = dinv[i];
        for (int c = tid; c < k; c += nt) {
            double v;
            if (c > i) v = 0.0;
            else if (c == i) v = di;
            else {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int e = c;
                for (; e + 3 < i; e += 4) {
                    s0 += A[i * k + e] * Li[e * k + c];
                    s1 += A[i * k + e + 1] * Li[(e + 1) * k + c];
                    s2 += A[i * k + e + 2] * Li[(e + 2) * k + c];
                    s3 += A[i * k + e + 3] * Li[(e + 3) * k + c];
                }
                for (; e < i; ++e) s0 += A[i * k + e] * Li[e * k + c];
                v = -((s0 + s1) + (s2 + s3)) * di;
            }
            Li[i * k + c] = v;
        }
        __syncthreads();
    }
    // G^-1 = Li^T Li into A (L is no longer needed).
    for (int e = tid; e < kk; e += nt) {
        const int c = e / k, d = e - c * k;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        if (act[c] && act[d]) {
            int q = c > d ? c : d;
            for (; q + 3 < k; q += 4) {
                s0 += Li[q * k + c] * Li[q * k + d];
                s1 += Li[(q + 1) * k + c] * Li[(q + 1) * k + d];
                s2 += Li[(q + 2) * k + c] * Li[(q + 2) * k + d];
                s3 += Li[(q + 3) * k + c] * Li[(q + 3) * k + d];
            }
            for (; q < k; ++q) s0 += Li[q * k + c] * Li[q * k + d];
        }
        A[e] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    for (int e = tid; e < kk; e += nt) {
        Ginv64[e] = A[e];
        GinvT[e] = (T)A[e];
    }
    if (tid == 0) {
        if (sing) atomicOr(status, ST_SINGULAR);
        if (nonfin) atomicOr(status, ST_NONFINITE);
    }
}

template <typename T>
cudaError_t launch_cholesky(const double* G, int k, double* Ginv64, T* GinvT,
                            unsigned* status, cudaStream_t st)
{
    const size_t kk8 = (size_t)k * k * sizeof(double);
    const size_t extra = (size_t)k * (sizeof(double) + sizeof(int)) + 16;
    const int li_smem = 2 * kk8 + extra <= 210 * 1024;
    const size_t smem = kk8 * (li_smem ? 2 : 1) + extra;
    int threads = k * k >= 1024 ? 1024 : ((k * k + 31) / 32) * 32;
    if (threads < 32) threads = 32;
    cholesky_kernel<T><<<1, threads, smem, st>>>(G, k, Ginv64, GinvT, status, li_smem);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dense rows x k (row-major) -> row-packed factor; entries that are not > 0
// after conversion to T are dropped; negative entries raise ST_BADINPUT,
// non-finite ones ST_NONFINITE.

template <typename Tin, typename T>
__global__ void dense_to_ell_kernel(const Tin* __restrict__ F, int64_t rows,
                                    int k, int ld, int32_t* cnt, int32_t* col,
                                    T* val, unsigned* status)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false, neg = false;
    for (int64_t r = w0; r < rows; r += nw) {
        int base = 0;
        for (int cc = 0; cc < k; cc += 32) {
            const int c = cc + lane;
            const Tin x = c < k ? F[r * k + c] : Tin(0);
            if (c < k && !isfinite((double)x)) bad = true;
            if (c < k && x < Tin(0)) neg = true;
            const T xv = (T)x;
            const bool keep = c < k && xv > T(0) && isfinite((double)x);
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = base + __popc(b & ((1u << lane) - 1u));
                col[r * ld + pos] = c;
                val[r * ld + pos] = xv;
            }
            base += __popc(b);
        }
        if (lane == 0) cnt[r] = base;
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    if (neg) atomicOr(status, ST_BADINPUT);
}

template <typename Tin, typename T>
cudaError_t launch_dense_to_ell(const Tin* F, int64_t rows, int k, EllDev out,
                                unsigned* status, cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    const int B = 256;
    int64_t grid = (rows * 32 + B - 1) / B;
    if (grid > 65535) grid = 65535;
    dense_to_ell_kernel<Tin, T><<<(unsigned)grid, B, 0, st>>>(
        F, rows, k, out.ld, out.cnt, out.col, static_cast<T*>(out.val), status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed-order two-level sums.

template <typename T>
__global__ void norm2_part_kernel(const T* __restrict__ v, int64_t count,
                                  double* part)
{
    __shared__ double red[32];
    const int64_t chunk = (count + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < count ? b0 + chunk : count;
    double s = 0.0;
    for (int64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
        const double x = (double)v[e];
        s += x * x;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void sum_parts_kernel(const double* part, int n, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
    }
}

template <typename T>
cudaError_t launch_norm2(const T* val, int64_t count, double* part,
                         int nparts, double* out, cudaStream_t st)
{
    norm2_part_kernel<T><<<nparts, 256, 0, st>>>(val, count, part);
    sum_parts_kernel<<<1, 32, 0, st>>>(part, nparts, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void ell_dot_part_kernel(int64_t rows, int ld, const int32_t* cnt,
                                    const int32_t* col, const T* val,
                                    const T* Y, int64_t ldy, double* part)
{
    __shared__ double red[32];
    const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < rows ? b0 + chunk : rows;
    double s = 0.0;
    for (int64_t r = b0 + threadIdx.x; r < b1; r += blockDim.x) {
        const int L = cnt[r];
        for (int q = 0; q < L; ++q)
            s += (double)val[r * ld + q] * (double)Y[r * ldy + col[r * ld + q]];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

template <typename T>
cudaError_t launch_ell_dot(int64_t rows, int k, EllDev F, const T* Y,
                           int64_t ldy, double* part, int nparts, double* out,
                           cudaStream_t st)
{
    (void)k;
    ell_dot_part_kernel<T><<<nparts, 256, 0, st>>>(rows, F.ld, F.cnt, F.col,
                                                   static_cast<const T*>(F.val), Y, ldy, part);
    sum_parts_kernel<<<1, 32, 0, st>>>(part, nparts, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout conversions used by the enforcement entry points.

template <typename T>
__global__ void ell_scatter_colmajor_kernel(int64_t rows, int ld,
                                            const int32_t* cnt,
                                            const int32_t* col, const T* val,
                                            T* Xt, int64_t ldx)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int L = cnt[r];
        for (int q = 0; q < L; ++q) Xt[(int64_t)col[r * ld + q] * ldx + r] = val[r * ld + q];
    }
}

template <typename T>
cudaError_t launch_ell_to_colmajor(int64_t rows, int k, EllDev F, T* Xt,
                                   int64_t ldx, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(Xt, 0, sizeof(T) * (size_t)k * ldx, st);
    if (e != cudaSuccess) return e;
    if (rows == 0) return cudaSuccess;
    int64_t grid = (rows + 255) / 256;
    if (grid > 65535) grid = 65535;
    ell_scatter_colmajor_kernel<T><<<(unsigned)grid, 256, 0, st>>>(
        rows, F.ld, F.cnt, F.col, static_cast<const T*>(F.val), Xt, ldx);
    return cudaGetLastError();
}

template <typename T>
__global__ void dense_to_colmajor_kernel(const T* __restrict__ X, int64_t rows,
                                         int k, int64_t ld, T* Xt,
                                         int64_t ldx, unsigned* status)
{
    bool bad = false;
    const int64_t total = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int c = (int)(e - r * k);
        const T x = X[r * ld + c];
        if (!isfinite((double)x)) bad = true;
        Xt[(int64_t)c * ldx + r] = x > T(0) ? x : T(0);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

template <typename T>
cudaError_t launch_dense_to_colmajor(const T* X, int64_t rows, int k,
                                     int64_t ld, T* Xt, int64_t ldx,
                                     unsigned* status, cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    int64_t grid = (rows * k + 255) / 256;
    if (grid > 65535) grid = 65535;
    dense_to_colmajor_kernel<T><<<(unsigned)grid, 256, 0, st>>>(X, rows, k, ld, Xt, ldx, status);
    return cudaGetLastError();
}

template <typename T>
__global__ void ell_to_dense_kernel(int64_t rows, int k, int eld,
                                    const int32_t* cnt, const int32_t* col,
                                    const T* val, T* X, int64_t ld)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < rows; r += nw) {
        for (int c = lane; c < k; c += 32) X[r * ld + c] = T(0);
        __syncwarp();
        const int L = cnt[r];
        for (int q = lane; q < L; q += 32) X[r * ld + col[r * eld + q]] = val[r * eld + q];
        __syncwarp();
    }
}

template <typename T>
cudaError_t launch_ell_to_dense(int64_t rows, int k, EllDev F, T* X,
                                int64_t ld, cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    int64_t grid = (rows * 32 + 255) / 256;
    if (grid > 65535) grid = 65535;
    ell_to_dense_kernel<T><<<(unsigned)grid, 256, 0, st>>>(
        rows, k, F.ld, F.cnt, F.col, static_cast<const T*>(F.val), X, ld);
    return cudaGetLastError();
}

cudaError_t setup_factor()
{
    cudaError_t e;
    e = cudaFuncSetAttribute(finalize_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(finalize_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(cholesky_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(cholesky_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

#define ESPNMF_INST(T)                                                                         \
    template cudaError_t launch_finalize<T>(int64_t, int, EllDev, EllDev, bool, bool, const T*, \
                                            int64_t, double*, double*, int, cudaStream_t);     \
    template cudaError_t launch_cholesky<T>(const double*, int, double*, T*, unsigned*,         \
                                            cudaStream_t);                                      \
    template cudaError_t launch_norm2<T>(const T*, int64_t, double*, int, double*, cudaStream_t); \
    template cudaError_t launch_ell_dot<T>(int64_t, int, EllDev, const T*, int64_t, double*,    \
                                           int, double*, cudaStream_t);                         \
    template cudaError_t launch_ell_to_colmajor<T>(int64_t, int, EllDev, T*, int64_t,          \
                                                   cudaStream_t);                               \
    template cudaError_t launch_dense_to_colmajor<T>(const T*, int64_t, int, int64_t, T*,      \
                                                     int64_t, unsigned*, cudaStream_t);         \
    template cudaError_t launch_ell_to_dense<T>(int64_t, int, EllDev, T*, int64_t, cudaStream_t);
ESPNMF_INST(float)
ESPNMF_INST(double)
#undef ESPNMF_INST

template cudaError_t launch_dense_to_ell<double, double>(const double*, int64_t, int, EllDev, unsigned*, cudaStream_t);
template cudaError_t launch_dense_to_ell<double, float>(const double*, int64_t, int, EllDev, unsigned*, cudaStream_t);
template cudaError_t launch_dense_to_ell<float, double>(const float*, int64_t, int, EllDev, unsigned*, cudaStream_t);
template cudaError_t launch_dense_to_ell<float, float>(const float*, int64_t, int, EllDev, unsigned*, cudaStream_t);

}  // namespace espnmf
