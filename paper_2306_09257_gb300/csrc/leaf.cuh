// Diagonal-block inversion shared by the float64 and the mixed path.
// (1) leaf_gj / leaf_gj_regs: Gauss-Jordan elimination with partial (row)
// pivoting of one NB x NB block.  (2) leaf128_recursive: the mixed path's
// 128 x 128 blocks, by the 2x2 Schur recursion in shared memory down to
// 32 x 32 Gauss-Jordan leaves held in registers.
// In (1), for the shared-memory form:  Thread t owns row t/4 and the columns sub + 4q
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

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// In-CTA recursive inverse of a 128 x 128 complex-symmetric fp32 block.
// The block stays in shared memory; the 2x2 Schur recursion of the global
// inversion (T = C Ai, D -= T B, D <- D^-1, V = D T, A += T^T V, C = -V,
// B = -V^T) runs down to 32 x 32 diagonal blocks, which are inverted by
// pivoted Gauss-Jordan on 8 warps with the rows in registers.  The products
// are CTA-wide fp32 GEMMs from shared memory.  512 threads, one CTA per block.
// ---------------------------------------------------------------------------
namespace rec {
constexpr int NT = 512;
constexpr int P128 = 130, P64 = 66, P32 = 34;  // padded pitches (float2)


// C = (ACC ? C : 0) + sgn * op(A) B, all H x H (H = 32 or 64), in shared memory
// (every block offset and pitch even, so column pairs are 16-byte aligned).
// Thread (rt, ct) computes rows rt + i * RT (i < RB) and the column pairs
// 2 (ct + q * CT) (q < NP), with the operands of step k + 1 loaded while
// step k is multiplied.
template <int H, bool TRANS_A, bool ACC>
__device__ void gemm(const float2 *A, int lda, const float2 *B, int ldb, float2 *C, int ldc, float sgn) {
    constexpr int CT = 16;                 // column-pair threads
    constexpr int RT = NT / CT;            // row threads (32)
    constexpr int RB = H / RT;             // rows per thread (2 for H = 64, 1 for H = 32)
    constexpr int NP = H / (2 * CT);       // column pairs per thread (2 or 1)
    const int t = threadIdx.x;
    const int rt = t / CT, ct = t % CT;
    float2 acc[RB][2 * NP];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int u = 0; u < 2 * NP; ++u) acc[i][u] = make_float2(0.f, 0.f);
    auto lda_ = [&](int k, int i) { const int r = rt + i * RT; return TRANS_A ? A[k * lda + r] : A[r * lda + k]; };
    auto ldb_ = [&](int k, int q) { return *reinterpret_cast<const float4 *>(B + k * ldb + 2 * (ct + q * CT)); };
    float2 a[RB];
    float4 b[NP];
#pragma unroll
    for (int i = 0; i < RB; ++i) a[i] = lda_(0, i);
#pragma unroll
    for (int q = 0; q < NP; ++q) b[q] = ldb_(0, q);
#pragma unroll 2
    for (int k = 0; k < H; ++k) {
        float2 an[RB];
        float4 bn[NP];
        const int kn = k + 1 < H ? k + 1 : k;
#pragma unroll
        for (int i = 0; i < RB; ++i) an[i] = lda_(kn, i);
#pragma unroll
        for (int q = 0; q < NP; ++q) bn[q] = ldb_(kn, q);
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 b0 = make_float2(b[q].x, b[q].y), b1 = make_float2(b[q].z, b[q].w);
                float2 &c0 = acc[i][2 * q], &c1 = acc[i][2 * q + 1];
                c0.x = fmaf(a[i].x, b0.x, fmaf(-a[i].y, b0.y, c0.x));
                c0.y = fmaf(a[i].x, b0.y, fmaf(a[i].y, b0.x, c0.y));
                c1.x = fmaf(a[i].x, b1.x, fmaf(-a[i].y, b1.y, c1.x));
                c1.y = fmaf(a[i].x, b1.y, fmaf(a[i].y, b1.x, c1.y));
            }
#pragma unroll
        for (int i = 0; i < RB; ++i) a[i] = an[i];
#pragma unroll
        for (int q = 0; q < NP; ++q) b[q] = bn[q];
    }
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float4 *c = reinterpret_cast<float4 *>(C + (rt + i * RT) * ldc + 2 * (ct + q * CT));
            float4 v = make_float4(sgn * acc[i][2 * q].x, sgn * acc[i][2 * q].y, sgn * acc[i][2 * q + 1].x,
                                   sgn * acc[i][2 * q + 1].y);
            if (ACC) {
                const float4 o = *c;
                v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
            }
            *c = v;
        }
}

// Pivoted Gauss-Jordan inverse of a 32 x 32 block (pitch ld) by NW warps
// (8 by default): lane i holds row i, warp w the columns CW w .. CW w + CW - 1
// (CW = 32 / NW), in registers.  Pivot rows are not swapped: step k takes the
// unused row p_k with the largest |a[p][k]| and eliminates column k from every
// other row, so that at the end storage row r holds row ipiv[r] of the inverse
// with its columns in pivot order: inv[ipiv[r]][p_c] = a[r][c].
// After each step every warp also stores its columns to a copy in shared
// memory (two copies, alternating by step), and the warp owning the next
// pivot column picks the pivot with one warp max-reduction over the key
// (|a[i][k]|^2 with its five low mantissa bits replaced by 31 - i, so ties go
// to the lowest row); after the step's one barrier of the NW warps each warp
// reads the pivot row and column from the copy.  `scr` holds 2 x 32 x LEAF_SP
// float2, 16-byte aligned.
constexpr int LEAF_SP = 34;

template <int NW>
static __device__ void leaf32t(float2 *a, int ld, float2 *scr, int *flags) {
    constexpr int CW = 32 / NW;  // columns per warp
    __shared__ int pp[2], piv[32];
    if (threadIdx.x >= 32 * NW) return;
    auto bar = [] { asm volatile("bar.sync 1, %0;" ::"n"(32 * NW) : "memory"); };
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2 x[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) x[j] = a[lane * ld + CW * w + j];
    // store this warp's columns to copy `b`; the owner of column k picks its pivot
    auto stage = [&](int b, int k, bool used) {
        float4 *dst = reinterpret_cast<float4 *>(scr + (b * 32 + lane) * LEAF_SP + CW * w);
#pragma unroll
        for (int j = 0; j < CW / 2; ++j) dst[j] = make_float4(x[2 * j].x, x[2 * j].y, x[2 * j + 1].x, x[2 * j + 1].y);
        if (w == k / CW) {
            const int kl = k % CW;
            float2 fk;
            if constexpr (CW == 8) {
                const float2 s0 = (kl & 1) ? x[1] : x[0], s1 = (kl & 1) ? x[3] : x[2];
                const float2 s2 = (kl & 1) ? x[5] : x[4], s3 = (kl & 1) ? x[7] : x[6];
                const float2 t0 = (kl & 2) ? s1 : s0, t1 = (kl & 2) ? s3 : s2;
                fk = (kl & 4) ? t1 : t0;
            } else {
                const float2 s0 = (kl & 1) ? x[1] : x[0], s1 = (kl & 1) ? x[3] : x[2];
                fk = (kl & 2) ? s1 : s0;
            }
            const unsigned bits = __float_as_uint(fk.x * fk.x + fk.y * fk.y);
            const unsigned key = used ? 0u : ((bits & ~31u) | (unsigned)(31 - lane));
            const unsigned best = __reduce_max_sync(0xffffffffu, key);
            if (lane == 0) {
                const int p = 31 - (int)(best & 31u);
                pp[b] = p;
                piv[k] = p;
            }
        }
    };
    bool used = false;
    int mystep = 0;
    stage(0, 0, false);
    bar();
    for (int k = 0; k < 32; ++k) {
        const int buf = k & 1;
        const int p = pp[buf];
        const float2 *cur = scr + buf * 32 * LEAF_SP;
        const float2 fk = cur[lane * LEAF_SP + k], d = cur[p * LEAF_SP + k];
        float2 rr[CW];
#pragma unroll
        for (int j = 0; j < CW / 2; ++j) {
            const float4 q = reinterpret_cast<const float4 *>(cur + p * LEAF_SP + CW * w)[j];
            rr[2 * j] = make_float2(q.x, q.y);
            rr[2 * j + 1] = make_float2(q.z, q.w);
        }
        const float den = d.x * d.x + d.y * d.y;
        if (threadIdx.x == 0 && (!(den > 0.f) || !isfinite(den))) atomicOr(flags, FLAG_SINGULAR);
        const float rd = __fdividef(1.f, den);
        const float2 inv = make_float2(d.x * rd, -d.y * rd);
        const bool isp = lane == p;
        if (isp) { used = true; mystep = k; }
        // pivot row: x <- x * inv; other rows: x <- x - f * (pivot row * inv)
        const float2 fe = isp ? make_float2(-1.f, 0.f) : fk;
        const float keep = isp ? 0.f : 1.f;
        const float2 ck = make_float2(-(fe.x * inv.x - fe.y * inv.y), -(fe.x * inv.y + fe.y * inv.x));
        const bool own = w == k / CW;
        const int kl = k % CW;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const float2 r = rr[j];
            const float2 n = make_float2(r.x * inv.x - r.y * inv.y, r.x * inv.y + r.y * inv.x);
            float2 v;
            v.x = fmaf(keep, x[j].x, -(fe.x * n.x - fe.y * n.y));
            v.y = fmaf(keep, x[j].y, -(fe.x * n.y + fe.y * n.x));
            x[j] = (own && j == kl) ? ck : v;
        }
        if (k + 1 < 32) stage(buf ^ 1, k + 1, used);
        bar();
    }
#pragma unroll
    for (int j = 0; j < CW; ++j) a[mystep * ld + piv[CW * w + j]] = x[j];
    bar();
}

static __device__ void leaf32(float2 *a, int ld, float2 *scr, int *flags) { leaf32t<8>(a, ld, scr, flags); }

// Symmetric 2x2 recursion on the n x n block at `a` (n = 32 or 64) with
// temporaries T, V (pitch P32) and the leaf scratch W.
template <int N>
__device__ void inv_sym(float2 *a, int ld, float2 *T, float2 *V, float2 *W, int *flags) {
    if constexpr (N == 32) {
        leaf32(a, ld, W, flags);
        __syncthreads();
    } else {
        constexpr int H = N / 2;
        float2 *A = a, *B = a + H, *C = a + H * ld, *D = a + H * ld + H;
        inv_sym<H>(A, ld, nullptr, nullptr, W, flags);
        gemm<H, false, false>(C, ld, A, ld, T, P32, 1.f);         // T = C Ai
        __syncthreads();
        gemm<H, false, true>(T, P32, B, ld, D, ld, -1.f);          // D -= T B
        __syncthreads();
        inv_sym<H>(D, ld, nullptr, nullptr, W, flags);
        gemm<H, false, false>(D, ld, T, P32, V, P32, 1.f);         // V = Si T
        __syncthreads();
        gemm<H, true, true>(T, P32, V, P32, A, ld, 1.f);           // A += T^T V
        for (int e = threadIdx.x; e < H * H; e += NT) {            // C = -V, B = -V^T
            const int r = e / H, cc = e % H;
            const float2 v = V[r * P32 + cc];
            C[r * ld + cc] = make_float2(-v.x, -v.y);
            B[cc * ld + r] = make_float2(-v.x, -v.y);
        }
        __syncthreads();
    }
}
}  // namespace rec

constexpr int rec_smem_bytes() {
    return (128 * rec::P128 + 2 * 64 * rec::P64 + 2 * 32 * rec::P32) * 8;
}

static __device__ void leaf128_recursive(float *re, float *im, long long ld, int *flags) {
    extern __shared__ __align__(16) unsigned char rec_smem[];
    // zero pivots of the recursive attempt are recorded here, not in `flags`:
    // the self-check below catches their effect and the fallback reports
    __shared__ int s_sing;
    if (threadIdx.x == 0) s_sing = 0;
    float2 *M = reinterpret_cast<float2 *>(rec_smem);
    float2 *T64 = M + 128 * rec::P128, *V64 = T64 + 64 * rec::P64;
    float2 *T32 = V64 + 64 * rec::P64, *V32 = T32 + 32 * rec::P32;
    for (int e = threadIdx.x; e < 128 * 128; e += rec::NT) {
        const int r = e >> 7, c = e & 127;
        const long long g = (long long)r * ld + c;
        M[r * rec::P128 + c] = make_float2(re[g], im[g]);
    }
    __syncthreads();
    // 128: split into 64 blocks (temps T64/V64), the 64 blocks use T32/V32
    {
        constexpr int H = 64;
        float2 *A = M, *B = M + H, *C = M + H * rec::P128, *D = M + H * rec::P128 + H;
        const int ld0 = rec::P128;
        rec::inv_sym<64>(A, ld0, T32, V32, V64, &s_sing);
        rec::gemm<H, false, false>(C, ld0, A, ld0, T64, rec::P64, 1.f);
        __syncthreads();
        rec::gemm<H, false, true>(T64, rec::P64, B, ld0, D, ld0, -1.f);
        __syncthreads();
        rec::inv_sym<64>(D, ld0, T32, V32, V64, &s_sing);
        rec::gemm<H, false, false>(D, ld0, T64, rec::P64, V64, rec::P64, 1.f);
        __syncthreads();
        rec::gemm<H, true, true>(T64, rec::P64, V64, rec::P64, A, ld0, 1.f);
        for (int e = threadIdx.x; e < H * H; e += rec::NT) {
            const int r = e / H, cc = e % H;
            const float2 v = V64[r * rec::P64 + cc];
            C[r * ld0 + cc] = make_float2(-v.x, -v.y);
            B[cc * ld0 + r] = make_float2(-v.x, -v.y);
        }
        __syncthreads();
    }
    // Self-check before the block is overwritten.  Pivoting stays inside the
    // 32 x 32 leaves, so a nearly singular leading sub-block of a block that
    // is itself well conditioned spoils the recursion; apply the computed
    // inverse to a fixed unit-modulus probe v and compare X (X^-1 v) with v.
    // Above 2e-5 relative residual (a sound block gives a few 1e-7) the block
    // is inverted again by Gauss-Jordan with pivoting over all 128 rows.
    __shared__ float2 s_y[128], s_v[128];
    __shared__ float s_part[rec::NT / 32];
    __shared__ int s_bad;
    {
        const int t = threadIdx.x, r = t >> 2, sub = t & 3;
        if (t < 128) {
            float sn, cs;
            sincosf(2.3999632f * (float)t, &sn, &cs);
            s_v[t] = make_float2(cs, sn);
        }
        __syncthreads();
        float2 y = make_float2(0.f, 0.f);
        for (int q = 0; q < 32; ++q) {
            const int c = sub + 4 * q;
            const float2 m = M[r * rec::P128 + c], v = s_v[c];
            y.x += m.x * v.x - m.y * v.y;
            y.y += m.x * v.y + m.y * v.x;
        }
        y.x += __shfl_xor_sync(0xffffffffu, y.x, 1);
        y.y += __shfl_xor_sync(0xffffffffu, y.y, 1);
        y.x += __shfl_xor_sync(0xffffffffu, y.x, 2);
        y.y += __shfl_xor_sync(0xffffffffu, y.y, 2);
        if (sub == 0) s_y[r] = y;
        __syncthreads();
        // row r of the original block, columns [32 sub, 32 sub + 32), 16-byte loads
        float2 z = make_float2(0.f, 0.f);
        const float *rr = re + (long long)r * ld + 32 * sub, *ri = im + (long long)r * ld + 32 * sub;
        if (((((uintptr_t)rr) | ((uintptr_t)ri)) & 15) == 0) {
            float4 a[8], b[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                a[q] = reinterpret_cast<const float4 *>(rr)[q];
                b[q] = reinterpret_cast<const float4 *>(ri)[q];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float xr[4] = {a[q].x, a[q].y, a[q].z, a[q].w}, xi[4] = {b[q].x, b[q].y, b[q].z, b[q].w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 yc = s_y[32 * sub + 4 * q + u];
                    z.x += xr[u] * yc.x - xi[u] * yc.y;
                    z.y += xr[u] * yc.y + xi[u] * yc.x;
                }
            }
        } else {
            for (int q = 0; q < 32; ++q) {
                const float xr = rr[q], xi = ri[q];
                const float2 yc = s_y[32 * sub + q];
                z.x += xr * yc.x - xi * yc.y;
                z.y += xr * yc.y + xi * yc.x;
            }
        }
        z.x += __shfl_xor_sync(0xffffffffu, z.x, 1);
        z.y += __shfl_xor_sync(0xffffffffu, z.y, 1);
        z.x += __shfl_xor_sync(0xffffffffu, z.x, 2);
        z.y += __shfl_xor_sync(0xffffffffu, z.y, 2);
        float e2 = 0.f;
        if (sub == 0) {
            const float2 v = s_v[r];
            e2 = (z.x - v.x) * (z.x - v.x) + (z.y - v.y) * (z.y - v.y);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
        if ((t & 31) == 0) s_part[t >> 5] = e2;
        __syncthreads();
        if (t == 0) {
            float tot = 0.f;
            for (int i = 0; i < rec::NT / 32; ++i) tot += s_part[i];
            s_bad = !(tot <= 4e-10f * 128.f);  // (2e-5)^2 |v|^2; also catches NaN
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) atomicAdd(flags + 1, 1);  // fallback count (flags[1])
        leaf_gj_regs<128>(re, im, ld, flags);
        return;
    }
    for (int e = threadIdx.x; e < 128 * 128; e += rec::NT) {
        const int r = e >> 7, c = e & 127;
        const long long g = (long long)r * ld + c;
        const float2 v = M[r * rec::P128 + c];
        re[g] = v.x;
        im[g] = v.y;
    }
}
