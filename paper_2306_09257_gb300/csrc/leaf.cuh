// Diagonal-block inversion shared by the float64 and the mixed path:
// Gauss-Jordan elimination with partial (row) pivoting of one NB x NB block
// in shared memory.  Thread t owns row t/4 and the columns sub + 4q
// (sub = t%4), so the 4 threads of a row sit in adjacent lanes and the
// pivot-row reads are conflict-free; rows are padded by 4 elements.
// Row interchanges of the sweep become column interchanges of the inverse,
// undone in reverse order at the end.
#pragma once
#include "apf_internal.h"

template <typename R>
struct Cplx;
template <>
struct Cplx<double> {
    using T = double2;
    __device__ static T mk(double a, double b) { return make_double2(a, b); }
};
template <>
struct Cplx<float> {
    using T = float2;
    __device__ static T mk(float a, float b) { return make_float2(a, b); }
};

// Planar (re, im) or interleaved global layout.
template <typename R, bool PLANAR>
struct LeafIO {
    R *re, *im;
    typename Cplx<R>::T *z;
    long long ld;
    __device__ typename Cplx<R>::T load(int r, int c) const {
        long long g = (long long)r * ld + c;
        if (PLANAR) return Cplx<R>::mk(re[g], im[g]);
        return z[g];
    }
    __device__ void store(int r, int c, typename Cplx<R>::T v) const {
        long long g = (long long)r * ld + c;
        if (PLANAR) { re[g] = v.x; im[g] = v.y; }
        else z[g] = v;
    }
};

template <typename R, int NB, bool PLANAR>
__device__ void leaf_gj(LeafIO<R, PLANAR> io, int *flags) {
    using T = typename Cplx<R>::T;
    constexpr int P = NB + 4;
    constexpr int NT = NB * 4;
    constexpr int Q = NB / 4;
    extern __shared__ __align__(16) unsigned char leaf_smem[];
    T *a = reinterpret_cast<T *>(leaf_smem);
    __shared__ T rowk[NB], colk[NB];
    __shared__ R mag[NB];
    __shared__ int piv[NB];
    __shared__ int s_p;
    const int t = threadIdx.x, i = t >> 2, sub = t & 3;
    for (int e = t; e < NB * NB; e += NT) {
        int r = e / NB, c = e % NB;  // NB is a compile-time power of two
        a[r * P + c] = io.load(r, c);
    }
    __syncthreads();
    if (t < NB) {
        T v = a[t * P];
        mag[t] = v.x * v.x + v.y * v.y;
    }
    __syncthreads();
    for (int k = 0; k < NB; ++k) {
        if (t < 32) {
            R best = (R)-1;
            int bi = k;
            for (int r = k + t; r < NB; r += 32) {
                R m = mag[r];
                if (m > best) { best = m; bi = r; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                R ob = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (t == 0) {
                s_p = bi;
                piv[k] = bi;
                if (!(best > (R)0) || !isfinite((double)best)) atomicOr(flags, FLAG_SINGULAR);
            }
        }
        __syncthreads();
        const int p = s_p;
        if (p != k && t < NB) {
            T x = a[k * P + t];
            a[k * P + t] = a[p * P + t];
            a[p * P + t] = x;
        }
        __syncthreads();
        if (t < NB) {
            T d = a[k * P + k];
            R den = d.x * d.x + d.y * d.y;
            T inv = Cplx<R>::mk(d.x / den, -d.y / den);
            T v = a[k * P + t];
            rowk[t] = (t == k) ? inv : Cplx<R>::mk(v.x * inv.x - v.y * inv.y, v.x * inv.y + v.y * inv.x);
            colk[t] = a[t * P + k];
        }
        __syncthreads();
        const T f = colk[i];
        T *row = a + i * P;
        if (i == k) {
#pragma unroll 8
            for (int q = 0; q < Q; ++q) row[sub + 4 * q] = rowk[sub + 4 * q];
        } else {
            R m1 = (R)-1;
#pragma unroll 8
            for (int q = 0; q < Q; ++q) {
                const int j = sub + 4 * q;
                T x = (j == k) ? Cplx<R>::mk(0, 0) : row[j];
                T rk = rowk[j];
                x.x -= f.x * rk.x - f.y * rk.y;
                x.y -= f.x * rk.y + f.y * rk.x;
                row[j] = x;
                if (j == k + 1) m1 = x.x * x.x + x.y * x.y;
            }
            if (((k + 1) & 3) == sub && k + 1 < NB) mag[i] = m1;
        }
        if (i == k && ((k + 1) & 3) == sub && k + 1 < NB) {
            T x = rowk[k + 1];
            mag[i] = x.x * x.x + x.y * x.y;
        }
        __syncthreads();
    }
    for (int k = NB - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k && t < NB) {
            T x = a[t * P + k];
            a[t * P + k] = a[t * P + p];
            a[t * P + p] = x;
        }
        __syncthreads();
    }
    for (int e = t; e < NB * NB; e += NT) {
        int r = e / NB, c = e % NB;
        io.store(r, c, a[r * P + c]);
    }
}

template <int NB>
constexpr int leaf_smem_bytes(int elem_bytes) {
    return NB * (NB + 4) * elem_bytes;
}

// Register-resident variant for the mixed path: thread t keeps row t/4,
// columns sub + 4q (q < NB/4) of the block in registers; the pivot row is the
// only data exchanged through shared memory.  Rows are never swapped: step k
// takes the largest unused |a[r][k]| as pivot row p_k and eliminates column k
// from every other row.  With piv[k] = p_k and ipiv[p_k] = k the inverse is
// inv[ipiv[r]][piv[c]] = a[r][c] (written out by a scatter at the end).
// For the non-pivot rows the update x[j] -= f * prow[j] also produces the
// new column-k entry -f / pivot, because prow[k] holds 1 + 1/pivot there and
// x[k] = f before the update.
template <int NB>
__device__ void leaf_gj_regs(float *re, float *im, long long ld, int *flags) {
    constexpr int Q = NB / 4;
    __shared__ float2 prow[NB];
    __shared__ float mag[NB];
    __shared__ int piv[NB], ipiv[NB];
    __shared__ int s_p;
    const int t = threadIdx.x, i = t >> 2, sub = t & 3, lane = t & 31;
    float2 a[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long g = (long long)i * ld + sub + 4 * q;
        a[q] = make_float2(re[g], im[g]);
    }
    bool used = false;
    float2 col = a[0];  // column k value, valid on the owner lanes (sub == k % 4)
    if (sub == 0) mag[i] = col.x * col.x + col.y * col.y;
    __syncthreads();
    for (int k = 0; k < NB; ++k) {
        if (t < 32) {
            float best = -1.f;
            int bi = 0;
#pragma unroll
            for (int r0 = 0; r0 < NB; r0 += 32) {
                float m = mag[r0 + t];
                if (m > best) { best = m; bi = r0 + t; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                float ob = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (t == 0) {
                s_p = bi;
                piv[k] = bi;
                ipiv[bi] = k;
                if (!(best > 0.f) || !isfinite(best)) atomicOr(flags, FLAG_SINGULAR);
            }
        }
        __syncthreads();
        const int p = s_p;
        const float2 f = make_float2(__shfl_sync(0xffffffffu, col.x, (lane & ~3) | (k & 3)),
                                     __shfl_sync(0xffffffffu, col.y, (lane & ~3) | (k & 3)));
        float2 pinv;
        {
            float den = f.x * f.x + f.y * f.y;
            pinv = make_float2(f.x / den, -f.y / den);
        }
        if (i == p) {
            used = true;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = sub + 4 * q;
                float2 x = (j == k) ? pinv
                                    : make_float2(a[q].x * pinv.x - a[q].y * pinv.y, a[q].x * pinv.y + a[q].y * pinv.x);
                a[q] = x;
                prow[j] = (j == k) ? make_float2(1.f + pinv.x, pinv.y) : x;
            }
        }
        __syncthreads();
        if (i != p) {
            const float nfx = -f.x, fy = f.y;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const float2 pr = prow[sub + 4 * q];
                float2 x = a[q];
                x.x = fmaf(nfx, pr.x, x.x);
                x.x = fmaf(fy, pr.y, x.x);
                x.y = fmaf(nfx, pr.y, x.y);
                x.y = fmaf(-fy, pr.x, x.y);
                a[q] = x;
            }
        }
        // next pivot column: a uniform switch on its register slot
        float2 nc = make_float2(0.f, 0.f);
        switch ((k + 1) >> 2) {
#define APF_NC_CASE(Z) case Z: if (Z < Q) nc = a[Z < Q ? Z : 0]; break;
            APF_NC_CASE(0) APF_NC_CASE(1) APF_NC_CASE(2) APF_NC_CASE(3) APF_NC_CASE(4) APF_NC_CASE(5)
            APF_NC_CASE(6) APF_NC_CASE(7) APF_NC_CASE(8) APF_NC_CASE(9) APF_NC_CASE(10) APF_NC_CASE(11)
            APF_NC_CASE(12) APF_NC_CASE(13) APF_NC_CASE(14) APF_NC_CASE(15) APF_NC_CASE(16) APF_NC_CASE(17)
            APF_NC_CASE(18) APF_NC_CASE(19) APF_NC_CASE(20) APF_NC_CASE(21) APF_NC_CASE(22) APF_NC_CASE(23)
            APF_NC_CASE(24) APF_NC_CASE(25) APF_NC_CASE(26) APF_NC_CASE(27) APF_NC_CASE(28) APF_NC_CASE(29)
            APF_NC_CASE(30) APF_NC_CASE(31)
#undef APF_NC_CASE
            default: break;
        }
        col = nc;
        if (k + 1 < NB && sub == ((k + 1) & 3)) mag[i] = used ? -1.f : nc.x * nc.x + nc.y * nc.y;
        __syncthreads();
    }
    const int r = ipiv[i];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long g = (long long)r * ld + piv[sub + 4 * q];
        re[g] = a[q].x;
        im[g] = a[q].y;
    }
}

// Faster register-resident variant: two barriers per elimination step.
//  * The argmax for the next pivot is reduced per warp during the update
//    (by the lanes that own the next column) and finished redundantly by
//    every thread from the per-warp partials.
//  * The pivot row is published unscaled; each thread folds 1/pivot into its
//    own row factor g = f / a_pk.  Column k of the published row carries
//    a_pk + 1, so x[k] - g (a_pk + 1) = -g, the new column-k entry.
template <int NB>
__device__ void leaf_gj_regs2(float *re, float *im, long long ld, int *flags) {
    constexpr int Q = NB / 4;
    constexpr int NW = NB * 4 / 32;  // warps
    __shared__ float2 prow[NB];
    __shared__ float pmag[2][NW];
    __shared__ int pidx[2][NW];
    __shared__ int piv[NB], ipiv[NB];
    const int t = threadIdx.x, i = t >> 2, sub = t & 3, lane = t & 31, warp = t >> 5;
    float2 a[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long g = (long long)i * ld + sub + 4 * q;
        a[q] = make_float2(re[g], im[g]);
    }
    bool used = false;
    float2 col = a[0];
    // warp-level partial argmax of |col|^2 over the owner lanes (sub == k % 4)
    auto publish = [&](int k, int buf) {
        float m = (sub == (k & 3) && !used) ? col.x * col.x + col.y * col.y : -1.f;
        int idx = i;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            float om = __shfl_down_sync(0xffffffffu, m, off);
            int oi = __shfl_down_sync(0xffffffffu, idx, off);
            if (om > m || (om == m && oi < idx)) { m = om; idx = oi; }
        }
        if (lane == 0) { pmag[buf][warp] = m; pidx[buf][warp] = idx; }
    };
    publish(0, 0);
    __syncthreads();
    for (int k = 0; k < NB; ++k) {
        const int buf = k & 1;
        float best = -1.f;
        int p = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            float m = pmag[buf][w];
            int idx = pidx[buf][w];
            if (m > best || (m == best && idx < p)) { best = m; p = idx; }
        }
        if (t == 0) {
            piv[k] = p;
            ipiv[p] = k;
            if (!(best > 0.f) || !isfinite(best)) atomicOr(flags, FLAG_SINGULAR);
        }
        const float2 f = make_float2(__shfl_sync(0xffffffffu, col.x, (lane & ~3) | (k & 3)),
                                     __shfl_sync(0xffffffffu, col.y, (lane & ~3) | (k & 3)));
        if (i == p) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = sub + 4 * q;
                prow[j] = (j == k) ? make_float2(a[q].x + 1.f, a[q].y) : a[q];
            }
        }
        __syncthreads();
        // pivot value from the published row (column k holds a_pk + 1)
        const float2 pk = prow[k];
        const float2 apk = make_float2(pk.x - 1.f, pk.y);
        const float den = apk.x * apk.x + apk.y * apk.y;
        const float2 pinv = make_float2(apk.x / den, -apk.y / den);
        float2 nc = make_float2(0.f, 0.f);
        if (i != p) {
            const float2 g = make_float2(f.x * pinv.x - f.y * pinv.y, f.x * pinv.y + f.y * pinv.x);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = sub + 4 * q;
                const float2 pr = prow[j];
                float2 x = a[q];
                x.x -= g.x * pr.x - g.y * pr.y;
                x.y -= g.x * pr.y + g.y * pr.x;
                a[q] = x;
                if (j == k + 1) nc = x;
            }
        } else {
            used = true;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = sub + 4 * q;
                float2 x = (j == k) ? pinv
                                    : make_float2(a[q].x * pinv.x - a[q].y * pinv.y, a[q].x * pinv.y + a[q].y * pinv.x);
                a[q] = x;
                if (j == k + 1) nc = x;
            }
        }
        col = nc;
        if (k + 1 < NB) publish(k + 1, buf ^ 1);
        __syncthreads();
    }
    const int r = ipiv[i];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long g = (long long)r * ld + piv[sub + 4 * q];
        re[g] = a[q].x;
        im[g] = a[q].y;
    }
}
