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
//   gram_inverse  FP64 inverse of the Gram matrix by the symmetric sweep
//                 operator (one CTA), used by the k x k solve.
//   conversions   dense -> row-packed, row-packed -> dense / column-major,
//                 ||A||^2 and the stand-alone <U, Y> reduction.
//
// Every reduction adds in a fixed order (per warp, then per block in warp
// order, then over blocks in block order), so all results are reproducible.
#include <float.h>

#include <algorithm>

#include "common.cuh"

namespace espnmf {

static __host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__device__ inline double warp_sum(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

constexpr int kEmitThreads = 256;   // 8 warps
constexpr int kSlots = 20;          // heavy-Gram register slots per thread

// Upper-triangle index of (c, d), c <= d, row by row.
__host__ __device__ inline int tri_index(int c, int d, int k) { return c * k - c * (c - 1) / 2 + (d - c); }

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
    uint4* rec;          // FP32: per-row records (cnt and the first pairs)
    uint32_t* nzmask;    // FP32: nonzero-row bitmask (or NULL)
    const int32_t* hslot;   // slot of the row in htab, or -1 (NULL: no table)
    T* htab;
    uint8_t* hnz;
    int ld, dld, heavy, SL;   // SL: staged pairs per lane (light rows)
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
           (size_t)W * align16((size_t)k * (k + 1) / 2 * 8) +
           (size_t)W * (align16((size_t)32 * SL * 4) + align16((size_t)32 * SL * sizeof(T))) +
           align16((size_t)kEmitThreads * 4) + align16((size_t)ld * 8) + 64;
}

template <typename T>
__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(EmitArgs<T> a)
{
    using K = typename KeyBits<T>::K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kEmitThreads / 32][4];
    __shared__ int wcnt[kEmitThreads / 32];
    const int k = a.k, ld = a.ld, SL = a.SL;
    const int W = blockDim.x >> 5;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* p = smem_raw;
    K* stau = reinterpret_cast<K*>(p);
    p += align16((size_t)a.nseg * sizeof(K));
    uint32_t* scut = reinterpret_cast<uint32_t*>(p);
    p += align16((size_t)a.nseg * 4);
    double* Gall = reinterpret_cast<double*>(p);
    p += (size_t)W * align16((size_t)k * (k + 1) / 2 * 8);
    int* stc_all = reinterpret_cast<int*>(p);
    p += (size_t)W * align16((size_t)32 * SL * 4);
    T* stv_all = reinterpret_cast<T*>(p);
    p += (size_t)W * align16((size_t)32 * SL * sizeof(T));
    int* hlist = reinterpret_cast<int*>(p);
    p += align16((size_t)kEmitThreads * 4);
    double* drow = reinterpret_cast<double*>(p);

    const size_t gstride = align16((size_t)k * (k + 1) / 2 * 8) / 8;
    double* G = Gall + (size_t)warp * gstride;
    int* stc = stc_all + (size_t)warp * (align16((size_t)32 * SL * 4) / 4);
    T* stv = stv_all + (size_t)warp * (align16((size_t)32 * SL * sizeof(T)) / sizeof(T));
    for (int c = tid; c < a.nseg; c += blockDim.x) {
        stau[c] = a.tau[c];
        scut[c] = a.cut[c];
    }
    for (int e = lane; e < k * (k + 1) / 2; e += 32) G[e] = 0.0;
    __syncthreads();

    const bool matrix = a.mode == TOPT_MATRIX;
    // blocks own whole 32-row words of the nonzero-row bitmask
    const int64_t chunk = ((a.rows + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
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
        bool nonzero = false;
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
                T* dr = a.dense + r * a.dld;
                for (int c = 0; c < ld; ++c) dr[c] = T(0);
                for (int j = 0; j < pos; ++j) dr[wc[j]] = wv[j];
            }
            if (a.hslot) {
                // a frequent row: its dense copy in the sparse product's table
                const int sl = a.hslot[r];
                if (sl >= 0) {
                    T* tr = a.htab + (int64_t)sl * ld;
                    for (int c = 0; c < ld; ++c) tr[c] = T(0);
                    for (int j = 0; j < pos; ++j) tr[wc[j]] = wv[j];
                    a.hnz[sl] = pos > 0 ? 1 : 0;
                }
            }
            nonzero = pos > 0;
            a.cnt[r] = pos;
            if constexpr (sizeof(T) == 4) {
                if (a.rec) {
                    // the first min(pos, 6) pairs: from this lane's staging,
                    // or from the row this thread has just written
                    unsigned x[2] = {(unsigned)pos, 0u};
                    unsigned v[6] = {0u, 0u, 0u, 0u, 0u, 0u};
                    for (int q = 0; q < pos && q < 6; ++q) {
                        const unsigned c = (unsigned)(q < SL ? stc[lane * SL + q] : wc[q]);
                        const float xv = (float)(q < SL ? stv[lane * SL + q] : wv[q]);
                        x[q / 3] |= c << (q < 3 ? 8 * (q + 1) : 8 * (q - 3));
                        v[q] = __float_as_uint(xv);
                    }
                    a.rec[2 * r] = make_uint4(x[0], v[0], v[1], v[2]);
                    a.rec[2 * r + 1] = make_uint4(x[1], v[3], v[4], v[5]);
                }
            }
            if (a.zero_old) a.cnt_old[r] = 0;
            nl = (hv && a.heavy_gram) ? 0 : pos;
        }
        __syncwarp();
        if (a.nzmask) {
            const unsigned word = __ballot_sync(0xffffffffu, nonzero);
            if (lane == 0) a.nzmask[base >> 5] = word;
        }
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
                    G[ca < cb ? tri_index(ca, cb, k) : tri_index(cb, ca, k)] += va * (double)jv[ib];
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
                for (int c = tid; c < k; c += blockDim.x) drow[c] = (double)a.dense[rr * a.dld + c];
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
        for (int w = 0; w < W; ++w) v += Gall[(size_t)w * gstride + tri_index(c, d, k)];
        a.gram_part[(size_t)tri_index(c, d, k) * P + blockIdx.x] = v;
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
        for (int w = 0; w < W; ++w) v += Gall[(size_t)w * gstride + tri_index(c, d, k)];
        a.gram_part[(size_t)tri_index(c, d, k) * P + blockIdx.x] = v;
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
    a.rec = cur.rec;
    a.nzmask = cur.nzmask;
    a.hslot = cur.h > 0 ? cur.hslot : nullptr;
    a.htab = static_cast<T*>(cur.htab);
    a.hnz = cur.hnz;
    a.ld = cur.ld;
    a.dld = cur.dld;
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
    // 8 warps unless shared memory says otherwise (two blocks per SM need
    // at most ~110 KB each); the heavy rows' Gram uses register slots when
    // they cover the triangle, else every row is staged for the pair loop
    int W = kEmitThreads / 32;
    size_t smem = 0;
    for (;;) {
        a.heavy_gram = cur.dense != nullptr && ntri <= kSlots * W * 32;
        a.SL = a.heavy_gram ? (cur.heavy - 1 > 0 ? cur.heavy - 1 : 1) : k;
        smem = emit_smem<T>(k, cur.ld, a.nseg, a.SL, W);
        if (smem <= 110 * 1024 || W == 1) break;
        --W;
    }
    emit_kernel<T><<<nblocks, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

__global__ void gram_reduce_kernel(const double* __restrict__ gram_part,
                                   const double* __restrict__ scal_part,
                                   int P, int Ps, int k, const double* __restrict__ diag_part,
                                   int Cd, bool pairs, double* G, double* scal,
                                   unsigned* counter, MetricsArgs m)
{
    // one warp per output: the upper-triangle Gram entries (partials
    // entry-major, P per entry), then the 4 scalars (Ps partials each); a
    // lane adds parts lane, lane+32, ... and the warp adds the lanes in a
    // fixed tree, so the sum is reproducible.  Diagonal entries also get the
    // Cd per-column partials of diag_part.
    const int ntri = k * (k + 1) / 2;
    const int kk = k * k;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w < ntri + 4) {
        const int np = w < ntri ? P : Ps;
        const double* src = w < ntri ? gram_part + (size_t)w * P : scal_part + (size_t)(w - ntri) * Ps;
        double v;
        // the partials are loaded eight at a time before they are added (in
        // the same order), so a lane waits for the L2 once per eight
        constexpr int U8 = 8;
        if (pairs) {
            // compensated pairs, added on the FP32 pipes, widened once
            const float2* sp = reinterpret_cast<const float2*>(src);
            DFloat acc;
            for (int p0 = lane; p0 < np; p0 += 32 * U8) {
                float2 b[U8];
#pragma unroll
                for (int u = 0; u < U8; ++u) {
                    const int p = p0 + 32 * u;
                    b[u] = p < np ? sp[p] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U8; ++u)
                    if (p0 + 32 * u < np) df_add(acc, b[u].x, b[u].y);
            }
            acc = df_warp_sum(acc);
            v = df_value(acc);
        } else {
            double s0 = 0.0, s1 = 0.0;
            int p = lane;
            for (; p + 32 * (U8 - 1) < np; p += 32 * U8) {
                double b[U8];
#pragma unroll
                for (int u = 0; u < U8; ++u) b[u] = src[p + 32 * u];
#pragma unroll
                for (int u = 0; u < U8; u += 2) {
                    s0 += b[u];
                    s1 += b[u + 1];
                }
            }
            for (; p + 32 < np; p += 64) {
                s0 += src[p];
                s1 += src[p + 32];
            }
            if (p < np) s0 += src[p];
            v = warp_sum(s0 + s1);
        }
        if (lane == 0) {
            if (w < ntri) {
                int c = 0, start = 0, rowlen = k;
                while (w >= start + rowlen) {
                    start += rowlen;
                    ++c;
                    --rowlen;
                }
                const int d = c + (w - start);
                if (c == d && diag_part) {
                    if (pairs) {
                        const float2* dp = reinterpret_cast<const float2*>(diag_part) + (size_t)c * Cd;
                        DFloat dg;
                        for (int j = 0; j < Cd; ++j) df_add(dg, dp[j].x, dp[j].y);
                        v += df_value(dg);
                    } else {
                        for (int j = 0; j < Cd; ++j) v += diag_part[(size_t)c * Cd + j];
                    }
                }
                G[c * k + d] = v;
                G[d * k + c] = v;
            } else {
                scal[w - ntri] = v;
            }
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
    for (int q0 = threadIdx.x; q0 < kk; q0 += 8 * blockDim.x) {
        double g[8], o[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * blockDim.x;
            g[u] = q < kk ? __ldcg(G + q) : 0.0;
            o[u] = q < kk ? m.G_other[q] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (q0 + u * (int)blockDim.x < kk) tr += g[u] * o[u];
    }
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

cudaError_t launch_gram_reduce(const double* gram_part, const double* scal_part, int nparts,
                               int nscal_parts, int k, const double* diag_part, int diag_parts,
                               bool pairs, double* G, double* scal, unsigned* counter,
                               MetricsArgs m, cudaStream_t st)
{
    const int B = 256;
    const int ntri = k * (k + 1) / 2;
    const int grid = ((ntri + 4) * 32 + B - 1) / B;
    gram_reduce_kernel<<<grid, B, 0, st>>>(gram_part, scal_part, nparts, nscal_parts, k,
                                           diag_part, diag_parts, pairs, G, scal, counter, m);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Survivor-driven emit (FP32 form, column mode).  The selector has marked
// every survivor in a per-row bitmask (bit c of row i: entry (i, c) is kept)
// and written the Gram diagonal; this pass reads each row's bits (and
// clears them for the next selection), writes the row's pairs from the
// candidate, its record, its nonzero bit, its dense copy (heavy rows) and
// its row of the frequent table, and accumulates in FP64 the Sec. 3.1 sums
// (||F_new - F_old||^2 over the union of the two supports, ||F_new||^2,
// ||F_old||^2, <F_new, Y>).  The off-diagonal Gram products of the rows
// with two or more nonzeros that are not frequent rows are added by one
// warp, row after row in row order, into the block's triangle; the frequent
// rows' products come from gram_table_kernel.  Work is proportional to the
// rows plus the survivors, not to rows x k.

struct EmitSArgs {
    const float* Xt;
    int64_t ldx;
    int64_t rows;
    int k;
    uint32_t* rowbits;
    int32_t* cnt;
    int32_t* col;
    float* val;
    float* dense;
    uint4* rec;
    uint32_t* nzmask;
    const int32_t* hslot;
    float* htab;
    uint8_t* hnz;
    int ld, dld, heavy;
    int32_t* cnt_old;
    const int32_t* col_old;
    const float* val_old;
    bool residual, zero_old;
    const float* Y;
    int64_t ldy;
    double* gram_part;   // [ntri][P], this kernel's blocks are columns [0, gridDim.x)
    double* scal_part;   // [4][gridDim.x]
    int P;
};

constexpr int kEmitSThreads = 512;
constexpr int kEmitSStage = 8;   // pairs per row staged in shared memory
constexpr int kLaneSurv = 8;     // rows with more survivors are written by a whole warp

template <int WD>
__global__ void __launch_bounds__(kEmitSThreads)
emit_s_kernel(EmitSArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DFloat* T = reinterpret_cast<DFloat*>(smem_raw);   // [ntri] compensated FP32 sums
    // the pairs of this round's rows (the first kEmitSStage of each), so
    // that the warp adding the off-diagonal products reads shared memory
    int2* stage = reinterpret_cast<int2*>(smem_raw + (((size_t)a.k * (a.k + 1) / 2 * sizeof(DFloat) + 15) & ~(size_t)15));
    __shared__ int wcount[kEmitSThreads / 32];
    __shared__ int list[kEmitSThreads];
    __shared__ int ccnt[kEmitSThreads / 32];
    __shared__ int lcnt[kEmitSThreads];               // this round's row counts
    __shared__ int clist[kEmitSThreads];              // this round's many-survivor rows
    __shared__ uint32_t cbits[kEmitSThreads][WD];     // their survivor bits
    __shared__ DFloat red[kEmitSThreads / 32][4];
    __shared__ float wold[kEmitSThreads / 32][kMaxK];   // a warp's old row, dense
    const int k = a.k, ld = a.ld;
    const int ntri = k * (k + 1) / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NW = blockDim.x >> 5;
    for (int e = tid; e < ntri; e += blockDim.x) T[e] = DFloat();
    // Warps own whole 32-row words of the nonzero-row bitmask, dealt out
    // round-robin over the blocks (word (rnd * NW + warp) * G + block), so
    // that rows with many survivors -- on text corpora the frequent terms,
    // which have the lowest ids -- spread over all blocks.
    const int64_t G = gridDim.x;
    const int64_t nwords = (a.rows + 31) / 32;
    auto word_of = [&](int64_t rnd, int w) -> int64_t { return (rnd * NW + w) * G + blockIdx.x; };
    // global row of local index lr = warp * 32 + lane of round rnd
    auto row_of = [&](int64_t rnd, int lr) -> int64_t { return word_of(rnd, lr >> 5) * 32 + (lr & 31); };
    // per-lane Sec. 3.1 sums in compensated FP32 (widened to FP64 at the end)
    DFloat s_diff, s_new, s_old, s_cross;

    for (int64_t rnd = 0; word_of(rnd, 0) < nwords; ++rnd) {
        const int64_t r = row_of(rnd, tid);
        const bool valid = r < a.rows;
        bool nonzero = false, offdiag = false;
        uint32_t bits[WD];
#pragma unroll
        for (int w = 0; w < WD; ++w) bits[w] = 0u;
        bool coop = false;
        if (valid) {
            uint32_t* bp = a.rowbits + r * WD;
#pragma unroll
            for (int w = 0; w < WD; ++w) bits[w] = bp[w];
#pragma unroll
            for (int w = 0; w < WD; ++w)
                if (bits[w]) bp[w] = 0u;
            int nb = 0;
#pragma unroll
            for (int w = 0; w < WD; ++w) nb += __popc(bits[w]);
            coop = nb > kLaneSurv;
            if (coop) {
                // written below by the whole warp
                const int sl = a.hslot ? a.hslot[r] : -1;
                nonzero = true;
                offdiag = sl < 0;
            }
        }
        if (valid && !coop) {
            int Lo = (a.residual || a.zero_old) ? a.cnt_old[r] : 0;
            if (!ESPNMF_CHECK(Lo <= ld, CHK_COUNT)) Lo = ld;
            const int32_t* co = a.col_old + r * ld;
            const float* vo = a.val_old + r * ld;
            int32_t* wc = a.col + r * ld;
            float* wv = a.val + r * ld;
            unsigned rx = 0u, rv0 = 0u, rv1 = 0u, rv2 = 0u;
            unsigned rx1 = 0u, rv3 = 0u, rv4 = 0u, rv5 = 0u;
            int pos = 0, q = 0;
#pragma unroll
            for (int w = 0; w < WD; ++w) {
                uint32_t mb = bits[w];
                while (mb) {
                    const int c = 32 * w + __ffs(mb) - 1;
                    mb &= mb - 1u;
                    if (!ESPNMF_CHECK(c < a.k, CHK_COLUMN)) continue;
                    const float x = a.Xt[(int64_t)c * a.ldx + r];
                    wc[pos] = c;
                    wv[pos] = x;
                    if (pos < kEmitSStage) stage[tid * kEmitSStage + pos] = make_int2(c, __float_as_int(x));
                    if (pos == 0) { rx |= (unsigned)c << 8; rv0 = __float_as_uint(x); }
                    else if (pos == 1) { rx |= (unsigned)c << 16; rv1 = __float_as_uint(x); }
                    else if (pos == 2) { rx |= (unsigned)c << 24; rv2 = __float_as_uint(x); }
                    else if (pos == 3) { rx1 |= (unsigned)c; rv3 = __float_as_uint(x); }
                    else if (pos == 4) { rx1 |= (unsigned)c << 8; rv4 = __float_as_uint(x); }
                    else if (pos == 5) { rx1 |= (unsigned)c << 16; rv5 = __float_as_uint(x); }
                    df_add_prod(s_new, x, x);
                    if (a.Y) df_add_prod(s_cross, x, a.Y[r * a.ldy + c]);
                    if (a.residual) {
                        while (q < Lo && co[q] < c) {
                            const float o = vo[q];
                            df_add_prod(s_old, o, o);
                            df_add_prod(s_diff, o, o);
                            ++q;
                        }
                        float o = 0.f;
                        if (q < Lo && co[q] == c) {
                            o = vo[q];
                            df_add_prod(s_old, o, o);
                            ++q;
                        }
                        df_add_sqdiff(s_diff, x, o);
                    }
                    ++pos;
                }
            }
            if (a.residual) {
                for (; q < Lo; ++q) {
                    const float o = vo[q];
                    df_add_prod(s_old, o, o);
                    df_add_prod(s_diff, o, o);
                }
            }
            a.cnt[r] = pos;
            lcnt[tid] = pos;
            if (a.rec) {
                a.rec[2 * r] = make_uint4(rx | (unsigned)pos, rv0, rv1, rv2);
                a.rec[2 * r + 1] = make_uint4(rx1, rv3, rv4, rv5);
            }
            if (a.zero_old) a.cnt_old[r] = 0;
            if (pos >= a.heavy && a.dense != nullptr) {
                float* dr = a.dense + r * a.dld;
                for (int c = 0; c < ld; ++c) dr[c] = 0.f;
                for (int j = 0; j < pos; ++j) dr[wc[j]] = wv[j];
            }
            const int sl = a.hslot ? a.hslot[r] : -1;
            if (sl >= 0) {
                float* tr = a.htab + (int64_t)sl * ld;
                for (int c = 0; c < ld; ++c) tr[c] = 0.f;
                for (int j = 0; j < pos; ++j) tr[wc[j]] = wv[j];
                a.hnz[sl] = pos > 0 ? 1 : 0;
            }
            nonzero = pos > 0;
            offdiag = pos >= 2 && sl < 0;
        }
        // rows with many survivors: listed in (warp, lane) order, then taken
        // one at a time by a whole warp (list entry j by warp j % NW): lane c
        // handles column c (and c + 32, ...), positions by prefix counts
        {
            const unsigned cb = __ballot_sync(0xffffffffu, coop);
            if (lane == 0) ccnt[warp] = __popc(cb);
            __syncthreads();
            int off = 0;
            for (int w = 0; w < warp; ++w) off += ccnt[w];
            if (coop) {
                const int j = off + __popc(cb & ((1u << lane) - 1u));
                clist[j] = tid;
#pragma unroll
                for (int w = 0; w < WD; ++w) cbits[j][w] = bits[w];
            }
        }
        int ctot = 0;
        for (int w = 0; w < NW; ++w) ctot += ccnt[w];
        __syncthreads();
        for (int j = warp; j < ctot; j += NW) {
            const int64_t rr = row_of(rnd, clist[j]);
            uint32_t bw[WD];
#pragma unroll
            for (int w = 0; w < WD; ++w) bw[w] = cbits[j][w];
            auto surv = [&](int c) -> bool {
                uint32_t wd = bw[0];
#pragma unroll
                for (int w = 1; w < WD; ++w)
                    if ((c >> 5) == w) wd = bw[w];
                return (wd >> (c & 31)) & 1u;
            };
            const int Lo = (a.residual || a.zero_old) ? a.cnt_old[rr] : 0;
            const int32_t* co = a.col_old + rr * ld;
            const float* vo = a.val_old + rr * ld;
            float* od = wold[warp];
            if (a.residual) {
                for (int c = lane; c < ld; c += 32) od[c] = 0.f;
                __syncwarp();
                for (int q = lane; q < Lo; q += 32) {
                    const int oc = co[q];
                    const float o = vo[q];
                    od[oc] = o;
                    df_add_prod(s_old, o, o);
                    if (!surv(oc)) df_add_prod(s_diff, o, o);
                }
                __syncwarp();
            }
            int32_t* wc = a.col + rr * ld;
            float* wv = a.val + rr * ld;
            const int sl = a.hslot ? a.hslot[rr] : -1;
            int before = 0, nb = 0;
#pragma unroll
            for (int w = 0; w < WD; ++w) nb += __popc(bw[w]);
            float* dr = nb >= a.heavy && a.dense != nullptr ? a.dense + rr * a.dld : nullptr;
            float* tr = sl >= 0 ? a.htab + (int64_t)sl * ld : nullptr;
            unsigned rx = (unsigned)nb, rx1 = 0u, rv[6] = {0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
            for (int w = 0; w < WD; ++w) {
                const int c = 32 * w + lane;
                const bool bit = (bw[w] >> lane) & 1u;
                const bool sv = bit && ESPNMF_CHECK(c < a.k, CHK_COLUMN);
                const int pos = before + __popc(bw[w] & ((1u << lane) - 1u));
                float x = 0.f;
                if (sv) {
                    x = a.Xt[(int64_t)c * a.ldx + rr];
                    wc[pos] = c;
                    wv[pos] = x;
                    df_add_prod(s_new, x, x);
                    if (a.Y) df_add_prod(s_cross, x, a.Y[rr * a.ldy + c]);
                    if (a.residual) df_add_sqdiff(s_diff, x, od[c]);
                }
                if (c < ld) {
                    if (dr) dr[c] = x;
                    if (tr) tr[c] = x;
                }
                // the record's first six pairs
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const unsigned who = __ballot_sync(0xffffffffu, sv && pos == q);
                    if (who) {
                        const int src = __ffs(who) - 1;
                        const unsigned cq = (unsigned)__shfl_sync(0xffffffffu, c, src);
                        const unsigned xq = __shfl_sync(0xffffffffu, __float_as_uint(x), src);
                        if (q < 3) rx |= cq << (8 * (q + 1));
                        else rx1 |= cq << (8 * (q - 3));
                        rv[q] = xq;
                    }
                }
                before += __popc(bw[w]);
            }
            if (dr)
                for (int c = 32 * WD + lane; c < a.dld; c += 32) dr[c] = 0.f;
            if (lane == 0) {
                a.cnt[rr] = nb;
                lcnt[clist[j]] = nb;
                if (a.rec) {
                    a.rec[2 * rr] = make_uint4(rx, rv[0], rv[1], rv[2]);
                    a.rec[2 * rr + 1] = make_uint4(rx1, rv[3], rv[4], rv[5]);
                }
                if (a.zero_old) a.cnt_old[rr] = 0;
                if (tr) a.hnz[sl] = 1;
            }
            __syncwarp();
        }
        if (a.nzmask) {
            const unsigned word = __ballot_sync(0xffffffffu, nonzero);
            const int64_t wd = word_of(rnd, warp);
            if (lane == 0 && wd < nwords) a.nzmask[wd] = word;
        }
        // this round's rows with off-diagonal products, in row order
        const unsigned ob = __ballot_sync(0xffffffffu, offdiag);
        if (lane == 0) wcount[warp] = __popc(ob);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < NW; ++w) {
            if (w < warp) off += wcount[w];
            tot += wcount[w];
        }
        if (offdiag) list[off + __popc(ob & ((1u << lane) - 1u))] = tid;
        __syncthreads();
        if (warp == 0) {
            for (int i = 0; i < tot; ++i) {
                const int lr = list[i];
                const int64_t rr = row_of(rnd, lr);
                const int L = lcnt[lr];
                if (L <= kEmitSStage) {
                    const int2* sp = stage + lr * kEmitSStage;
                    for (int ia = 0; ia + 1 < L; ++ia) {
                        const int2 pa = sp[ia];
                        const float va = __int_as_float(pa.y);
                        const int ib = ia + 1 + lane;
                        if (ib < L) {
                            const int2 pb = sp[ib];
                            df_add_prod(T[tri_index(pa.x, pb.x, k)], va, __int_as_float(pb.y));
                        }
                        __syncwarp();
                    }
                } else {
                    // a long row (rare): its pairs from global memory
                    const int32_t* cr = a.col + rr * ld;
                    const float* vr = a.val + rr * ld;
                    for (int ia = 0; ia + 1 < L; ++ia) {
                        const int ca = cr[ia];
                        const float va = vr[ia];
                        for (int ib = ia + 1 + lane; ib < L; ib += 32)
                            df_add_prod(T[tri_index(ca, cr[ib], k)], va, vr[ib]);
                        __syncwarp();
                    }
                }
            }
        }
        // the next round's first barrier orders warp 0's reads of `list`
        // before the list is rewritten
    }
    __syncthreads();
    // partials as compensated pairs (float2 in the double slots); the
    // reduction widens them once
    float2* gp = reinterpret_cast<float2*>(a.gram_part);
    for (int e = tid; e < ntri; e += blockDim.x)
        gp[(size_t)e * a.P + blockIdx.x] = make_float2(T[e].hi, T[e].lo);
    DFloat sc[4] = {s_diff, s_new, s_old, s_cross};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        sc[j] = df_warp_sum(sc[j]);
        if (lane == 0) red[warp][j] = sc[j];
    }
    __syncthreads();
    if (tid < 4) {
        DFloat sum;
        for (int w = 0; w < NW; ++w) df_add(sum, red[w][tid].hi, red[w][tid].lo);
        reinterpret_cast<float2*>(a.scal_part)[(size_t)tid * gridDim.x + blockIdx.x] =
            make_float2(sum.hi, sum.lo);
    }
}

cudaError_t launch_emit_s(const float* Xt, int64_t ldx, int64_t rows, int k, uint32_t* rowbits,
                          EllDev cur, EllDev old, bool residual, const float* Y, int64_t ldy,
                          double* gram_part, double* scal_part, int nblocks, int P,
                          cudaStream_t st)
{
    EmitSArgs a;
    a.Xt = Xt;
    a.ldx = ldx;
    a.rows = rows;
    a.k = k;
    a.rowbits = rowbits;
    a.cnt = cur.cnt;
    a.col = cur.col;
    a.val = static_cast<float*>(cur.val);
    a.dense = static_cast<float*>(cur.dense);
    a.rec = cur.rec;
    a.nzmask = cur.nzmask;
    a.hslot = cur.h > 0 ? cur.hslot : nullptr;
    a.htab = static_cast<float*>(cur.htab);
    a.hnz = cur.hnz;
    a.ld = cur.ld;
    a.dld = cur.dld;
    a.heavy = cur.heavy;
    a.cnt_old = old.cnt;
    a.col_old = old.col;
    a.val_old = static_cast<const float*>(old.val);
    a.residual = residual && old.cnt != nullptr;
    a.zero_old = old.cnt != nullptr;
    a.Y = Y;
    a.ldy = ldy;
    a.gram_part = gram_part;
    a.scal_part = scal_part;
    a.P = P;
    const size_t smem = (((size_t)k * (k + 1) / 2 * sizeof(DFloat) + 15) & ~(size_t)15) +
                        (size_t)kEmitSThreads * kEmitSStage * sizeof(int2);
    const int wd = (k + 31) / 32;
    switch (wd) {
    case 1: emit_s_kernel<1><<<nblocks, kEmitSThreads, smem, st>>>(a); break;
    case 2: emit_s_kernel<2><<<nblocks, kEmitSThreads, smem, st>>>(a); break;
    case 3: emit_s_kernel<3><<<nblocks, kEmitSThreads, smem, st>>>(a); break;
    case 4: emit_s_kernel<4><<<nblocks, kEmitSThreads, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Off-diagonal Gram products of the frequent rows, from their dense table
// (h rows of ld floats): block b adds the products of its share of the
// rows into its partial column pcol0 + b (entry-major, upper triangle,
// diagonal entries 0: the selector provides the diagonal).  Thread tid owns
// the entries e = tid + 256 s in FP64 registers.
constexpr int kTableRows = 16;   // table rows staged per pass

template <int S>
__global__ void __launch_bounds__(256)
gram_table_kernel(const float* __restrict__ htab, const uint8_t* __restrict__ hnz, int h,
                  int k, int ld, double* gram_part, int P, int pcol0)
{
    __shared__ float rowd[kTableRows][kMaxK];
    const int tid = threadIdx.x;
    const int ntri = k * (k + 1) / 2;
    int cd[S];
    DFloat acc[S];
    {
        int e0 = tid, c = 0, rowlen = k, start = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int e = e0 + s * 256;
            if (e < ntri) {
                while (e >= start + rowlen) {
                    start += rowlen;
                    ++c;
                    --rowlen;
                }
                const int d = c + (e - start);
                cd[s] = c < d ? ((c << 16) | d) : -1;
            } else {
                cd[s] = -1;
            }
        }
    }
    const int r0 = (int)((int64_t)h * blockIdx.x / gridDim.x);
    const int r1 = (int)((int64_t)h * (blockIdx.x + 1) / gridDim.x);
    // up to kTableRows rows at a time: one load round trip and two barriers
    // per pass (a zero row contributes zeros)
    for (int rb = r0; rb < r1; rb += kTableRows) {
        const int nr = r1 - rb < kTableRows ? r1 - rb : kTableRows;
        __syncthreads();
        for (int e = tid; e < nr * k; e += blockDim.x) {
            const int q = e / k, c = e - q * k;
            rowd[q][c] = hnz[rb + q] ? htab[(int64_t)(rb + q) * ld + c] : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < nr; ++q) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (cd[s] >= 0) df_add_prod(acc[s], rowd[q][cd[s] >> 16], rowd[q][cd[s] & 0xffff]);
        }
    }
    float2* gp = reinterpret_cast<float2*>(gram_part);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int e = tid + s * 256;
        if (e < ntri) gp[(size_t)e * P + pcol0 + blockIdx.x] = make_float2(acc[s].hi, acc[s].lo);
    }
}

ESPNMF_CHECK_READER(check_flags_factor)

cudaError_t launch_gram_table(const EllDev& F, int k, double* gram_part, int P, int pcol0,
                              int nblocks, cudaStream_t st)
{
    if (F.h <= 0) return cudaSuccess;
    const int ntri = k * (k + 1) / 2;
    const int S = (ntri + 255) / 256;
    const float* tab = static_cast<const float*>(F.htab);
    if (S <= 4) gram_table_kernel<4><<<nblocks, 256, 0, st>>>(tab, F.hnz, F.h, k, F.ld, gram_part, P, pcol0);
    else if (S <= 8) gram_table_kernel<8><<<nblocks, 256, 0, st>>>(tab, F.hnz, F.h, k, F.ld, gram_part, P, pcol0);
    else if (S <= 16) gram_table_kernel<16><<<nblocks, 256, 0, st>>>(tab, F.hnz, F.h, k, F.ld, gram_part, P, pcol0);
    else if (S <= 33) gram_table_kernel<33><<<nblocks, 256, 0, st>>>(tab, F.hnz, F.h, k, F.ld, gram_part, P, pcol0);
    else return cudaErrorInvalidValue;
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
// FP64 inverse of the Gram matrix G = F^T F in one CTA, by the symmetric
// sweep operator (Gauss-Jordan elimination with diagonal pivots, in place on
// the upper triangle).  Sweeping pivot p with d = a_pp maps
//   a_ij -> a_ij - a_ip a_pj / d   (i, j != p),
//   a_ip -> a_ip / d,   a_pp -> -1 / d,
// and after every index has been swept the array holds -G^-1.  The pivot d
// at step p is the p-th Schur complement pivot, i.e. the d_p of G = L D L^T
// (the square of the Cholesky diagonal), so the Cholesky pivot test applies:
// d_p <= 64 eps max_j G_jj raises ST_SINGULAR.  An index whose diagonal is
// exactly 0 belongs to an all-zero factor column; it is never swept and its
// row and column stay 0, which gives the minimum-norm solution.
//
// FP64 is slow on this GPU (a warp-wide FMA holds a sub-partition's FP64
// pipe for tens of cycles), so the kernel does the minimum k^3 / 2 FMAs and
// keeps the pipe busy:
//   * every thread owns a segment of one row of the upper triangle (row i,
//     up to E consecutive columns, segments cut at multiples of E) for the
//     whole factorisation, in registers: per step it reads pv[i] once and
//     does E independent FMAs;
//   * a step has two phases between barriers: the pivot row is scaled by
//     1/d (prs), then every entry is updated; the owners of the next pivot's
//     row publish it (pv, double-buffered) and the owners of diagonal
//     entries publish the diagonal (double-buffered);
//   * the next pivot's reciprocal is computed during the update phase by a
//     warp of its own (the last one), from the published diagonal and the
//     same FMA the entry's owner performs, so its FP64 latency chain is off
//     the critical path.
// The reciprocal comes from an FP32 seed refined by two FP64 Newton steps.

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

constexpr int kInvMaxWork = 512 - 32;    // threads that own entries

// Segments of the upper triangle with segment length E: row i holds columns
// [i, k), cut at multiples of E.
__host__ __device__ inline int inv_row_segments(int i, int k, int E)
{
    return (k - 1) / E - i / E + 1;
}

__host__ __device__ inline int inv_segments(int k, int E)
{
    int n = 0;
    for (int i = 0; i < k; ++i) n += inv_row_segments(i, k, E);
    return n;
}

struct InvSmem {
    size_t pv, prs, diag, alist, total;
};

__host__ __device__ inline InvSmem inv_smem(int k)
{
    InvSmem s;
    s.pv = 0;                                                   // 2 x k doubles
    s.prs = align16(s.pv + 2 * (size_t)k * sizeof(double));    // k doubles
    s.diag = align16(s.prs + (size_t)k * sizeof(double));      // 2 x k doubles
    s.alist = align16(s.diag + 2 * (size_t)k * sizeof(double)); // k + 1 ints
    s.total = align16(s.alist + ((size_t)k + 1) * sizeof(int));
    return s;
}

template <typename T, int E>
__global__ void __launch_bounds__(512)
gram_inverse_kernel(const double* __restrict__ G, int k, double* Ginv64,
                    T* GinvT, unsigned* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const InvSmem lay = inv_smem(k);
    double* pvb = reinterpret_cast<double*>(smem_raw + lay.pv);     // [2][k]
    double* prs = reinterpret_cast<double*>(smem_raw + lay.prs);    // [k]
    double* diagb = reinterpret_cast<double*>(smem_raw + lay.diag); // [2][k]
    int* alist = reinterpret_cast<int*>(smem_raw + lay.alist);      // active indices
    __shared__ double rbuf[2];
    __shared__ double maxdiag;
    __shared__ int na, sing, nonfin;
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    const int nwork = nt - 32;               // the last warp computes reciprocals
    const bool recip_warp = tid >= nwork;

    // this thread's segment: row si, columns [sj, sj + sn)
    int si = -1, sj = 0, sn = 0;
    if (!recip_warp) {
        int base = 0;
        for (int i = 0; i < k; ++i) {
            const int ns = inv_row_segments(i, k, E);
            if (tid < base + ns) {
                const int s = tid - base;
                si = i;
                sj = s == 0 ? i : (i / E + s) * E;
                const int end = min(k, (sj / E + 1) * E);
                sn = end - sj;
                break;
            }
            base += ns;
        }
    }
    if (tid == 0) {
        double md = 0.0;
        int nf = 0, cnt = 0;
        for (int j = 0; j < k; ++j) {
            const double d = G[(size_t)j * k + j];
            if (!isfinite(d)) nf = 1;
            if (d != 0.0 && isfinite(d)) {
                alist[cnt++] = j;
                if (d > md) md = d;
            }
        }
        alist[cnt] = -1;
        na = cnt;
        maxdiag = md;
        sing = 0;
        nonfin = nf;
    }
    double a[E];
#pragma unroll
    for (int e = 0; e < E; ++e) a[e] = (si >= 0 && e < sn) ? G[(size_t)si * k + sj + e] : 0.0;
    __syncthreads();
    const double tol = 64.0 * DBL_EPSILON * maxdiag;

    // step 0 inputs: the first pivot's row, the diagonal, its reciprocal
    const int p0 = na > 0 ? alist[0] : 0;
    for (int x = tid; x < k; x += nt) {
        pvb[x] = na > 0 ? G[(size_t)(x < p0 ? x : p0) * k + (x < p0 ? p0 : x)] : 0.0;
        diagb[x] = G[(size_t)x * k + x];
    }
    if (tid == 0 && na > 0) {
        const double d = G[(size_t)p0 * k + p0];
        const bool bad = !(d > tol);
        if (bad) sing = 1;
        rbuf[0] = recip_fp64(bad ? 1.0 : d);
    }
    __syncthreads();

    for (int s = 0; s < na; ++s) {
        const int p = alist[s];
        const int qn = alist[s + 1];            // next pivot, -1 after the last
        const double* pv = pvb + (s & 1) * k;
        double* pvn = pvb + ((s + 1) & 1) * k;
        const double* dg = diagb + (s & 1) * k;
        double* dgn = diagb + ((s + 1) & 1) * k;
        const double r = rbuf[s & 1];
        for (int x = tid; x < k; x += nt) prs[x] = pv[x] * r;
        __syncthreads();
        if (si >= 0) {
            if (si == p) {
                // the pivot's own row: a_pj -> a_pj / d, a_pp -> -1 / d
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e < sn) a[e] = sj + e == p ? -r : prs[sj + e];
            } else {
                const double pvi = pv[si];
                const double pri = prs[si];
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e < sn) a[e] = sj + e == p ? pri : fma(-pvi, prs[sj + e], a[e]);
            }
            if (si == qn) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e < sn) pvn[sj + e] = a[e];
            } else if (qn >= sj && qn < sj + sn) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (sj + e == qn) pvn[si] = a[e];
            }
            if (sj == si) dgn[si] = a[0];
        } else if (tid == nwork && qn >= 0) {
            // same FMA as the owner of (qn, qn): bitwise the same pivot
            const double d = fma(-pv[qn], prs[qn], dg[qn]);
            const bool bad = !(d > tol);
            if (bad) sing = 1;
            rbuf[(s + 1) & 1] = recip_fp64(bad ? 1.0 : d);
        }
        __syncthreads();
    }
    // the array holds -G^-1 on the active indices and 0 elsewhere
    if (si >= 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if (e >= sn) continue;
            const int i = si, j = sj + e;
            const double v = -a[e];
            Ginv64[(size_t)i * k + j] = v;
            Ginv64[(size_t)j * k + i] = v;
            GinvT[(size_t)i * k + j] = (T)v;
            GinvT[(size_t)j * k + i] = (T)v;
        }
    }
    if (tid == 0) {
        if (sing) atomicOr(status, ST_SINGULAR);
        if (nonfin) atomicOr(status, ST_NONFINITE);
    }
}

template <typename T, int E>
static cudaError_t launch_inverse_e(const double* G, int k, double* Ginv64, T* GinvT,
                                    unsigned* status, cudaStream_t st, int nseg)
{
    const int threads = (nseg + 31) / 32 * 32 + 32;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = inv_smem(k).total;
    cfg.stream = st;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;   // ahead of the concurrent SpMM's pending blocks
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gram_inverse_kernel<T, E>, G, k, Ginv64, GinvT, status);
}

template <typename T>
cudaError_t launch_gram_inverse(const double* G, int k, double* Ginv64, T* GinvT,
                                unsigned* status, cudaStream_t st)
{
    // the shortest segments that fit the block
    int n = inv_segments(k, 4);
    if (n <= kInvMaxWork) return launch_inverse_e<T, 4>(G, k, Ginv64, GinvT, status, st, n);
    n = inv_segments(k, 8);
    if (n <= kInvMaxWork) return launch_inverse_e<T, 8>(G, k, Ginv64, GinvT, status, st, n);
    n = inv_segments(k, 16);
    if (n <= kInvMaxWork) return launch_inverse_e<T, 16>(G, k, Ginv64, GinvT, status, st, n);
    n = inv_segments(k, 32);
    if (n <= kInvMaxWork) return launch_inverse_e<T, 32>(G, k, Ginv64, GinvT, status, st, n);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Fixed-order two-level sums.

template <typename T>
__global__ void norm2_part_kernel(const T* __restrict__ v, int64_t count,
                                  const uint2* __restrict__ v2, int64_t count2,
                                  const uint2* __restrict__ v3, int64_t count3,
                                  double* part)
{
    __shared__ double red[32];
    const int64_t total = count + count2 + count3;
    const int64_t chunk = (total + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < total ? b0 + chunk : total;
    double s = 0.0;
    for (int64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
        double x;
        if (e < count) x = (double)v[e];
        else if (e < count + count2) x = (double)__uint_as_float(v2[e - count].y);
        else x = (double)__uint_as_float(v3[e - count - count2].y);
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
cudaError_t launch_norm2(const T* val, int64_t count, const uint2* ent2, int64_t count2,
                         const uint2* ent3, int64_t count3, double* part, int nparts,
                         double* out, cudaStream_t st)
{
    if (ent2 == nullptr) count2 = 0;
    if (ent3 == nullptr) count3 = 0;
    norm2_part_kernel<T><<<nparts, 256, 0, st>>>(val, count, ent2, count2, ent3, count3, part);
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

// A caller's BF16 factor as FP32: the BF16 bits are the high half of the
// FP32 word, so the conversion is exact.
__global__ void bf16_to_f32_kernel(const uint16_t* __restrict__ x, int64_t count,
                                   float* __restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = __uint_as_float((uint32_t)x[e] << 16);
}

cudaError_t launch_bf16_to_f32(const uint16_t* x, int64_t count, float* y, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>((count + 255) / 256, 4096);
    bf16_to_f32_kernel<<<(unsigned)grid, 256, 0, st>>>(x, count, y);
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
    // emit_s needs at most k(k+1)/2 compensated pairs (k <= 128: 66 KB) and
    // the 32 KB stage, beside its static arrays
    auto es = [&](auto kern) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return r;
    };
    e = es(emit_s_kernel<1>);
    if (e == cudaSuccess) e = es(emit_s_kernel<2>);
    if (e == cudaSuccess) e = es(emit_s_kernel<3>);
    if (e == cudaSuccess) e = es(emit_s_kernel<4>);
    return e;
}

#define ESPNMF_INST(T)                                                                         \
    template cudaError_t launch_emit<T>(const T*, int64_t, int64_t, int, int, const void*,       \
                                        const uint32_t*, EllDev, EllDev, bool, const T*,       \
                                        int64_t, double*, double*, int, cudaStream_t);          \
    template cudaError_t launch_gram_inverse<T>(const double*, int, double*, T*, unsigned*,         \
                                            cudaStream_t);                                      \
    template cudaError_t launch_norm2<T>(const T*, int64_t, const uint2*, int64_t, const uint2*, \
                                         int64_t, double*, int, double*, cudaStream_t);         \
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
