// k_factor.cu -- everything that happens to a factor after its selection:
//
//   emit          row-wise pass over the projected candidate and the
//                 selector's thresholds: writes the new factor's rows in
//                 column order (and dense copies of heavy rows), zeroes the
//                 old buffer's counts, and leaves per-block FP64 partial sums
//                 of its Gram matrix F^T F (the "U^T U" / "V^T V" of Alg. 2
//                 steps 1 and 3), of ||F_new - F_old||^2, ||F_new||^2,
//                 ||F_old||^2 (Sec. 3.1 residual) and of <U, A V> (the cross
//                 term of the error identity).
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

__device__ inline double warp_sum(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

constexpr int kEmitThreads = 128;   // 4 warps
constexpr int kSlots = 40;          // heavy-Gram register slots per thread

template <typename T>
struct EmitArgs {
    const T* Xt;
    int64_t ldx;
    int64_t rows;
    int k, mode, nseg;
    const typename KeyBits<T>::K* tau;
    const uint32_t* cut;
    int32_t* cnt;
    int32_t* col;
    T* val;
    T* dense;
    int ld, heavy, SL;   // SL: staged pairs per lane (light rows)
    bool heavy_gram;     // heavy rows' Gram by register slots
    int32_t* cnt_old;
    const int32_t* col_old;
    const T* val_old;
    bool residual, zero_old;
    const T* Y;
    int64_t ldy;
    double* gram_part;   // [k*k][gridDim.x]
    double* scal_part;   // [4][gridDim.x]
};

template <typename T>
static size_t emit_smem(int k, int ld, int nseg, int SL, int W)
{
    using K = typename KeyBits<T>::K;
    return align16((size_t)nseg * sizeof(K)) + align16((size_t)nseg * 4) +
           (size_t)W * align16((size_t)k * k * 8) +
           (size_t)W * (align16((size_t)32 * SL * 4) + align16((size_t)32 * SL * sizeof(T))) +
           align16((size_t)kEmitThreads * 4) + align16((size_t)ld * 8) + 64;
}

template <typename T>
__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(EmitArgs<T> a)
{
    using K = typename KeyBits<T>::K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][4];
    __shared__ int wcnt[4];
    const int k = a.k, ld = a.ld, SL = a.SL;
    const int W = blockDim.x >> 5;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* p = smem_raw;
    K* stau = reinterpret_cast<K*>(p);
    p += align16((size_t)a.nseg * sizeof(K));
    uint32_t* scut = reinterpret_cast<uint32_t*>(p);
    p += align16((size_t)a.nseg * 4);
    double* Gall = reinterpret_cast<double*>(p);
    p += (size_t)W * align16((size_t)k * k * 8);
    int* stc_all = reinterpret_cast<int*>(p);
    p += (size_t)W * align16((size_t)32 * SL * 4);
    T* stv_all = reinterpret_cast<T*>(p);
    p += (size_t)W * align16((size_t)32 * SL * sizeof(T));
    int* hlist = reinterpret_cast<int*>(p);
    p += align16((size_t)kEmitThreads * 4);
    double* drow = reinterpret_cast<double*>(p);

    const size_t gstride = align16((size_t)k * k * 8) / 8;
    double* G = Gall + (size_t)warp * gstride;
    int* stc = stc_all + (size_t)warp * (align16((size_t)32 * SL * 4) / 4);
    T* stv = stv_all + (size_t)warp * (align16((size_t)32 * SL * sizeof(T)) / sizeof(T));
    for (int c = tid; c < a.nseg; c += blockDim.x) {
        stau[c] = a.tau[c];
        scut[c] = a.cut[c];
    }
    for (int e = lane; e < k * k; e += 32) G[e] = 0.0;
    __syncthreads();

    const bool matrix = a.mode == TOPT_MATRIX;
    const int64_t chunk = (a.rows + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < a.rows ? b0 + chunk : a.rows;
    double s_diff = 0.0, s_new = 0.0, s_old = 0.0, s_cross = 0.0;

    for (int64_t base = b0 + (int64_t)warp * 32; base < b1; base += (int64_t)W * 32) {
        const int64_t r = base + lane;
        const bool valid = r < b1;
        auto keep = [&](int c, T x) -> bool {
            const int sg = matrix ? 0 : c;
            const uint32_t ix = matrix ? (uint32_t)(r * k + c) : (uint32_t)r;
            return keep_entry<T>(x, stau[sg], scut[sg], ix);
        };
        int nl = 0;
        if (valid) {
            int pos = 0, q = 0;
            const int Lo = (a.residual || a.zero_old) ? a.cnt_old[r] : 0;
            const int32_t* co = a.col_old + r * ld;
            const T* vo = a.val_old + r * ld;
            int oc = (a.residual && Lo > 0) ? co[0] : k;
            int32_t* wc = a.col + r * ld;
            T* wv = a.val + r * ld;
            // one pass over the row's k candidates, eight loads in flight
            for (int c0 = 0; c0 < k; c0 += 8) {
                T xs[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    xs[u] = c0 + u < k ? a.Xt[(int64_t)(c0 + u) * a.ldx + r] : T(0);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int c = c0 + u;
                    if (c >= k) break;
                    const T x = xs[u];
                    const bool kp = keep(c, x);
                    if (kp) {
                        wc[pos] = c;
                        wv[pos] = x;
                        s_new += (double)x * (double)x;
                        if (a.Y) s_cross += (double)x * (double)a.Y[r * a.ldy + c];
                        if (pos < SL) {
                            stc[lane * SL + pos] = c;
                            stv[lane * SL + pos] = x;
                        }
                        ++pos;
                    }
                    if (a.residual) {
                        double o = 0.0;
                        if (oc == c) {
                            o = (double)vo[q];
                            ++q;
                            oc = q < Lo ? co[q] : k;
                            s_old += o * o;
                        }
                        if (kp || o != 0.0) {
                            const double d = (kp ? (double)x : 0.0) - o;
                            s_diff += d * d;
                        }
                    }
                }
            }
            const bool hv = pos >= a.heavy && a.dense != nullptr;
            if (hv) {
                // dense copy of a heavy row, from the pairs just written
                T* dr = a.dense + r * ld;
                for (int c = 0; c < ld; ++c) dr[c] = T(0);
                for (int j = 0; j < pos; ++j) dr[wc[j]] = wv[j];
            }
            a.cnt[r] = pos;
            if (a.zero_old) a.cnt_old[r] = 0;
            nl = (hv && a.heavy_gram) ? 0 : pos;
        }
        __syncwarp();
        // Gram of the light rows: a row's pairs (ia <= ib) across the lanes,
        // into the upper triangle (slot min*k + max); slots are distinct
        // within a row, rows follow each other.
        for (int j = 0; j < 32; ++j) {
            const int Lj = __shfl_sync(0xffffffffu, nl, j);
            const int* jc = stc + j * SL;
            const T* jv = stv + j * SL;
            for (int ia = 0; ia < Lj; ++ia) {
                const int ca = jc[ia];
                const double va = (double)jv[ia];
                for (int ib = ia + lane; ib < Lj; ib += 32) {
                    const int cb = jc[ib];
                    G[ca < cb ? ca * k + cb : cb * k + ca] += va * (double)jv[ib];
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // Gram of the heavy rows from their dense copies: thread tid owns the
    // upper-triangle entries e = tid + NT * s, in registers.
    const int ntri = k * (k + 1) / 2;
    const int NT = blockDim.x;
    int cd[kSlots];
    double acc[kSlots];
    {
        // (c, d) of entry e, c <= d, entries ordered by c then d
        int e0 = tid, c = 0, rowlen = k, start = 0;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            acc[s] = 0.0;
            const int e = e0 + s * NT;
            if (e < ntri) {
                while (e >= start + rowlen) {
                    start += rowlen;
                    ++c;
                    --rowlen;
                }
                cd[s] = (c << 16) | (c + (e - start));
            } else {
                cd[s] = -1;
            }
        }
    }
    if (a.heavy_gram && a.dense != nullptr) {
        for (int64_t base = b0; base < b1; base += NT) {
            const int64_t r = base + tid;
            const bool f = r < b1 && a.cnt[r] >= a.heavy;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = 0, nh = 0;
            for (int w = 0; w < W; ++w) {
                if (w < warp) off += wcnt[w];
                nh += wcnt[w];
            }
            if (f) hlist[off + __popc(bal & ((1u << lane) - 1u))] = (int)r;
            __syncthreads();
            for (int h = 0; h < nh; ++h) {
                const int64_t rr = hlist[h];
                for (int c = tid; c < k; c += blockDim.x) drow[c] = (double)a.dense[rr * ld + c];
                __syncthreads();
#pragma unroll
                for (int s = 0; s < kSlots; ++s)
                    if (cd[s] >= 0) acc[s] += drow[cd[s] >> 16] * drow[cd[s] & 0xffff];
                __syncthreads();
            }
        }
    }
    // block partial, entry-major, the upper triangle mirrored
    const int P = gridDim.x;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        if (cd[s] < 0) continue;
        const int c = cd[s] >> 16, d = cd[s] & 0xffff;
        double v = acc[s];
        for (int w = 0; w < W; ++w) v += Gall[(size_t)w * gstride + c * k + d];
        a.gram_part[(size_t)(c * k + d) * P + blockIdx.x] = v;
        if (c != d) a.gram_part[(size_t)(d * k + c) * P + blockIdx.x] = v;
    }
    // entries beyond the register slots (only for k too large for them)
    for (int e = kSlots * NT + tid; e < ntri; e += NT) {
        int c = 0, start = 0, rowlen = k;
        while (e >= start + rowlen) {
            start += rowlen;
            ++c;
            --rowlen;
        }
        const int d = c + (e - start);
        double v = 0.0;
        for (int w = 0; w < W; ++w) v += Gall[(size_t)w * gstride + c * k + d];
        a.gram_part[(size_t)(c * k + d) * P + blockIdx.x] = v;
        if (c != d) a.gram_part[(size_t)(d * k + c) * P + blockIdx.x] = v;
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
    if (tid < 4) {
        double sum = 0.0;
        for (int w = 0; w < W; ++w) sum += red[w][tid];
        a.scal_part[(size_t)tid * P + blockIdx.x] = sum;
    }
}

template <typename T>
cudaError_t launch_emit(const T* Xt, int64_t ldx, int64_t rows, int k, int mode,
                        const void* tau, const uint32_t* cut, EllDev cur, EllDev old,
                        bool residual, const T* Y, int64_t ldy, double* gram_part,
                        double* scal_part, int nblocks, cudaStream_t st)
{
    using K = typename KeyBits<T>::K;
    EmitArgs<T> a;
    a.Xt = Xt;
    a.ldx = ldx;
    a.rows = rows;
    a.k = k;
    a.mode = mode;
    a.nseg = mode == TOPT_MATRIX ? 1 : k;
    a.tau = static_cast<const K*>(tau);
    a.cut = cut;
    a.cnt = cur.cnt;
    a.col = cur.col;
    a.val = static_cast<T*>(cur.val);
    a.dense = static_cast<T*>(cur.dense);
    a.ld = cur.ld;
    a.heavy = cur.heavy;
    const int ntri = k * (k + 1) / 2;
    a.cnt_old = old.cnt;
    a.col_old = old.col;
    a.val_old = static_cast<const T*>(old.val);
    a.residual = residual && old.cnt != nullptr;
    a.zero_old = old.cnt != nullptr;
    a.Y = Y;
    a.ldy = ldy;
    a.gram_part = gram_part;
    a.scal_part = scal_part;
    // 4 warps unless shared memory says otherwise; the heavy rows' Gram
    // uses register slots when they cover the triangle, else every row is
    // staged for the pair loop
    int W = 4;
    size_t smem = 0;
    for (;;) {
        a.heavy_gram = cur.dense != nullptr && ntri <= kSlots * W * 32;
        a.SL = a.heavy_gram ? (cur.heavy - 1 > 0 ? cur.heavy - 1 : 1) : k;
        smem = emit_smem<T>(k, cur.ld, a.nseg, a.SL, W);
        if (smem <= 200 * 1024 || W == 1) break;
        --W;
    }
    emit_kernel<T><<<nblocks, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

__global__ void gram_reduce_kernel(const double* __restrict__ gram_part,
                                   const double* __restrict__ scal_part,
                                   int P, int k, double* G, double* scal,
                                   unsigned* counter, MetricsArgs m)
{
    // one warp per output: the k*k Gram entries, then the 4 scalars; a lane
    // adds parts lane, lane+32, ... and the warp adds the lanes in a fixed
    // tree, so the sum is reproducible
    const int kk = k * k;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < kk + 4) {
        const double* src = w < kk ? gram_part + (size_t)w * P : scal_part + (size_t)(w - kk) * P;
        double s0 = 0.0, s1 = 0.0;
        int p = lane;
        for (; p + 32 < P; p += 64) {
            s0 += src[p];
            s1 += src[p + 32];
        }
        if (p < P) s0 += src[p];
        const double v = warp_sum(s0 + s1);
        if (lane == 0) {
            if (w < kk) G[w] = v;
            else scal[w - kk] = v;
        }
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
    if (lane == 0) red[threadIdx.x >> 5] = tr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
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
    const int grid = ((k * k + 4) * 32 + B - 1) / B;
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
// FP64 inverse of the Gram matrix through its square-root-free Cholesky
// factorisation G = L D L^T (L unit lower triangular), in one CTA:
//   G^-1 = L^-T D^-1 L^-1.
// An index whose diagonal is exactly 0 belongs to an all-zero factor column:
// it is taken out (identity row/column during the factorisation, zero
// row/column in the inverse), which gives the minimum-norm solution.  A pivot
// d_j <= 64 eps max_j G_jj elsewhere raises ST_SINGULAR (d_j is the square
// of the Cholesky diagonal, so this is the LL^T pivot test).
// FP64 on this GPU has a long latency, so the column loop has one barrier
// per column and takes pivot reciprocals from an FP32 seed refined by two
// FP64 Newton steps.

__device__ __forceinline__ double recip_fp64(double d)
{
    const double ad = fabs(d);
    if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
    double x = (double)__frcp_rn((float)d);
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}

template <typename T>
__global__ void __launch_bounds__(256)
cholesky_kernel(const double* __restrict__ G, int k, double* Ginv64,
                T* GinvT, unsigned* status, int w_in_smem)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* A = reinterpret_cast<double*>(smem_raw);                 // k*k
    double* W = w_in_smem ? A + (size_t)k * k : Ginv64;               // k*k: L^-1
    double* dinv = A + (size_t)k * k * (w_in_smem ? 2 : 1);          // k
    int* act = reinterpret_cast<int*>(dinv + k);
    __shared__ double maxdiag;
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
    // L D L^T, lower triangle of A: after step j, A[i][j] (i > j) = l_ij
    for (int j = 0; j < k; ++j) {
        const double d0 = A[j * k + j];
        const bool bad = act[j] && !(d0 > tol);
        const double r = recip_fp64(bad ? 1.0 : d0);
        // trailing update with the unscaled column: a_il -= a_ij a_lj / d_j
        const int nrem = k - j - 1;
        for (int e = tid; e < nrem * nrem; e += nt) {
            const int ii = e / nrem, ll = e - ii * nrem;
            if (ll <= ii) {
                const int i = j + 1 + ii, l = j + 1 + ll;
                A[i * k + l] -= A[i * k + j] * (A[l * k + j] * r);
            }
        }
        __syncthreads();   // column j is read by everyone; scale it now
        if (tid == 0) {
            if (bad) sing = 1;
            dinv[j] = r;
            A[j * k + j] = 1.0;
        }
        for (int i = j + 1 + tid; i < k; i += nt) A[i * k + j] *= r;
    }
    __syncthreads();
    // W = L^-1 (unit lower), row by row; dot products over four accumulators
    for (int i = 0; i < k; ++i) {
        for (int c = tid; c < k; c += nt) {
            double v;
            if (c > i) v = 0.0;
            else if (c == i) v = 1.0;
            else {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int e = c;
                for (; e + 3 < i; e += 4) {
                    s0 += A[i * k + e] * W[e * k + c];
                    s1 += A[i * k + e + 1] * W[(e + 1) * k + c];
                    s2 += A[i * k + e + 2] * W[(e + 2) * k + c];
                    s3 += A[i * k + e + 3] * W[(e + 3) * k + c];
                }
                for (; e < i; ++e) s0 += A[i * k + e] * W[e * k + c];
                v = -((s0 + s1) + (s2 + s3));
            }
            W[i * k + c] = v;
        }
        __syncthreads();
    }
    // G^-1 = W^T D^-1 W on the upper triangle, mirrored into A
    const int ntri = k * (k + 1) / 2;
    for (int e = tid; e < ntri; e += nt) {
        int c = 0, start = 0, rowlen = k;
        while (e >= start + rowlen) {
            start += rowlen;
            ++c;
            --rowlen;
        }
        const int d = c + (e - start);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        if (act[c] && act[d]) {
            int q = d;
            for (; q + 3 < k; q += 4) {
                s0 += W[q * k + c] * dinv[q] * W[q * k + d];
                s1 += W[(q + 1) * k + c] * dinv[q + 1] * W[(q + 1) * k + d];
                s2 += W[(q + 2) * k + c] * dinv[q + 2] * W[(q + 2) * k + d];
                s3 += W[(q + 3) * k + c] * dinv[q + 3] * W[(q + 3) * k + d];
            }
            for (; q < k; ++q) s0 += W[q * k + c] * dinv[q] * W[q * k + d];
        }
        const double v = (s0 + s1) + (s2 + s3);
        A[c * k + d] = v;
        A[d * k + c] = v;
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
    const int w_smem = 2 * kk8 + extra <= 210 * 1024;
    const size_t smem = kk8 * (w_smem ? 2 : 1) + extra;
    int threads = k * k >= 256 ? 256 : ((k * k + 31) / 32) * 32;
    if (threads < 32) threads = 32;
    cholesky_kernel<T><<<1, threads, smem, st>>>(G, k, Ginv64, GinvT, status, w_smem);
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

template <typename Tin, typename T>
__global__ void dense_to_colmajor_kernel(const Tin* __restrict__ X, int64_t rows,
                                         int k, int64_t ld, T* Xt,
                                         int64_t ldx, unsigned* status,
                                         bool reject_negative)
{
    bool bad = false, neg = false;
    const int64_t total = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int c = (int)(e - r * k);
        const Tin x = X[r * ld + c];
        if (!isfinite((double)x)) bad = true;
        if (x < Tin(0)) neg = true;
        const T v = (T)x;
        Xt[(int64_t)c * ldx + r] = v > T(0) ? v : T(0);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    if (neg && reject_negative) atomicOr(status, ST_BADINPUT);
}

template <typename Tin, typename T>
cudaError_t launch_dense_to_colmajor(const Tin* X, int64_t rows, int k,
                                     int64_t ld, T* Xt, int64_t ldx,
                                     unsigned* status, bool reject_negative,
                                     cudaStream_t st)
{
    if (rows == 0) return cudaSuccess;
    int64_t grid = (rows * k + 255) / 256;
    if (grid > 65535) grid = 65535;
    dense_to_colmajor_kernel<Tin, T><<<(unsigned)grid, 256, 0, st>>>(X, rows, k, ld, Xt, ldx,
                                                                      status, reject_negative);
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
    e = cudaFuncSetAttribute(emit_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(emit_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(cholesky_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(cholesky_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

#define ESPNMF_INST(T)                                                                         \
    template cudaError_t launch_emit<T>(const T*, int64_t, int64_t, int, int, const void*,       \
                                        const uint32_t*, EllDev, EllDev, bool, const T*,       \
                                        int64_t, double*, double*, int, cudaStream_t);          \
    template cudaError_t launch_cholesky<T>(const double*, int, double*, T*, unsigned*,         \
                                            cudaStream_t);                                      \
    template cudaError_t launch_norm2<T>(const T*, int64_t, double*, int, double*, cudaStream_t); \
    template cudaError_t launch_ell_dot<T>(int64_t, int, EllDev, const T*, int64_t, double*,    \
                                           int, double*, cudaStream_t);                         \
    template cudaError_t launch_ell_to_colmajor<T>(int64_t, int, EllDev, T*, int64_t,          \
                                                   cudaStream_t);                               \
    template cudaError_t launch_ell_to_dense<T>(int64_t, int, EllDev, T*, int64_t, cudaStream_t);
ESPNMF_INST(float)
ESPNMF_INST(double)
#undef ESPNMF_INST

template cudaError_t launch_dense_to_colmajor<double, double>(const double*, int64_t, int, int64_t, double*, int64_t, unsigned*, bool, cudaStream_t);
template cudaError_t launch_dense_to_colmajor<double, float>(const double*, int64_t, int, int64_t, float*, int64_t, unsigned*, bool, cudaStream_t);
template cudaError_t launch_dense_to_colmajor<float, double>(const float*, int64_t, int, int64_t, double*, int64_t, unsigned*, bool, cudaStream_t);
template cudaError_t launch_dense_to_colmajor<float, float>(const float*, int64_t, int, int64_t, float*, int64_t, unsigned*, bool, cudaStream_t);

}  // namespace espnmf
