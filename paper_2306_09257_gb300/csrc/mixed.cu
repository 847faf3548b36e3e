// Mixed-precision slab elimination and float64 iterative refinement.
//
// The slab Schur blocks X_j and their inverses G_j are held in float32
// (separate real / imaginary planes).  Every product runs on the tensor cores
// (tc_gemm.cu) with operands split into bf16 planes: two planes and three
// products ("bf16x3") for the elimination and the field sweeps, three planes
// and six products for the gradient contraction.  Accuracy is then won back
// by float64 iterative refinement of the slab fields:
//     r = R - K E (float64 5-point stencil + boundary circulants),
//     E <- E + Khat^-1 r,
// where Khat^-1 is the block-LU solve with the stored low-precision G_j.
#include "apf_internal.h"
#include "tc_gemm.h"
#include "leaf.cuh"

#include <algorithm>
#include <complex>
#include <stdio.h>
#include <stdlib.h>
#include <vector>

struct MixedWork {
    int nsplit_elim = 2, nsplit_grad = 3, leaf = 128, leaf_variant = 0;
    float *Xre = nullptr, *Xim = nullptr;            // n x n working block
    float *Tre = nullptr, *Tim = nullptr;            // recursion scratch (n*n/2 each)
    float *Vre = nullptr, *Vim = nullptr;
    __nv_bfloat16 *PA = nullptr, *PB = nullptr;      // operand packs
    long long pa_elems = 0, pb_elems = 0;
    __nv_bfloat16 *GP = nullptr;                     // packed G_j: h of them, or seg_rows when recomputing
    long long gp_stride = 0;
    // Recomputation of the slab Schur blocks (seg_rows > 0): the rows are cut
    // into segments of seg_rows; only the packed inverses of one segment are
    // held (GP slot j - start of j's segment), plus the float32 G_{c-1} at every
    // segment start c > 0 (checkpoint s-1 for segment s), from which a
    // segment's inverses are recomputed when a sweep needs them.
    int seg_rows = 0, nseg = 1, seg_loaded = -1;
    float *CK = nullptr;                             // (nseg - 1) checkpoints, 2 n^2 floats each
    // Symmetric random butterfly transform of every slab block before its
    // inversion (bfly = 1): X' = U^T X U, G = U X'^-1 U^T with a depth-2
    // recursive butterfly U; BW holds its 2 n random diagonal entries.
    int bfly = 0;
    float *BW = nullptr;
    float *O32 = nullptr;                            // GEMM output planes, 2 * max(ncol, n_out) * nx
    double2 *r = nullptr, *delta = nullptr;          // refinement buffers (h*ncol*nx)
    double2 *cb = nullptr, *ct = nullptr;            // circulant products on the boundary rows
    double *rnorm = nullptr;                         // ||R_c||^2, ||r_c||^2
    int km = 0;                                      // GMRES(km) refinement (0: plain refinement)
    double2 *KV = nullptr, *KZ = nullptr;            // Krylov basis (km+1 fields) and preconditioned vectors (km)
    double2 *kdot = nullptr, *ky = nullptr;          // Gram-Schmidt coefficients (km+1)*km*ncol, update km*ncol
    double *knrm = nullptr;                          // ||W_c||^2 per Arnoldi step, km*ncol
    std::vector<void *> allocs;
};

namespace {
struct Bat;
}
int recompute_segment_b(const Bat &bt, int seg, cudaStream_t s);

namespace {

// Per-design pointers of a batch of designs (entry blockIdx.z, or blockIdx.x
// for the one-CTA-per-block leaf kernel); a single design uses entry 0.
template <typename T>
struct Tab {
    T v[TC_MAX_BATCH];
};

__device__ __forceinline__ void split_bf16(float x, int nsplit, __nv_bfloat16 *o) {
    __nv_bfloat16 h0 = __float2bfloat16_rn(x);
    o[0] = h0;
    if (nsplit > 1) {
        float x1 = x - __bfloat162float(h0);
        __nv_bfloat16 h1 = __float2bfloat16_rn(x1);
        o[1] = h1;
        if (nsplit > 2) o[2] = __float2bfloat16_rn(x1 - __bfloat162float(h1));
    }
}

// Pack a complex float32 planar matrix into bf16 split planes.
// Logical element v(r, k) = trans ? src[k][r] : src[r][k], r < R, k < K.
// layoutB = 0 (A operand): row r = [Re v(r,:), Im v(r,:)].
// layoutB = 1 (B operand of C = A B, r indexing C's columns):
//   row r = [Re v(r,:), -Im v(r,:)], row R + r = [Im v(r,:), Re v(r,:)].
struct PackJob {
    const float *re, *im;
    long long ld;
    int R, K, trans, layoutB, nsplit;
    __nv_bfloat16 *out;
    long long kp, plane_pitch;
};
// Up to N pack jobs per launch (blockIdx.z): the two operands of one product,
// or those of the same product for every design of a batch.
template <int N>
struct PackJobsN {
    PackJob j[N];
};
constexpr int MAX_JOBS = 2 * TC_MAX_BATCH;

// Tile: 32 rows x 64 k; thread (tx, ty) handles k = k0 + 2 tx, +1 (bf16x2 stores).
template <int N>
__global__ void __launch_bounds__(256) k_pack32(const __grid_constant__ PackJobsN<N> jobs) {
    const PackJob &J = jobs.j[blockIdx.z];
    __shared__ float tre[32][65], tim[32][65];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
    if (r0 >= J.R || k0 >= J.K) return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (!J.trans) {
        for (int i = ty; i < 32; i += 8) {
            int r = r0 + i;
            for (int kk = tx; kk < 64; kk += 32) {
                int k = k0 + kk;
                float a = 0.f, b = 0.f;
                if (r < J.R && k < J.K) { a = J.re[(long long)r * J.ld + k]; b = J.im[(long long)r * J.ld + k]; }
                tre[i][kk] = a; tim[i][kk] = b;
            }
        }
    } else {
        for (int kk = ty; kk < 64; kk += 8) {
            int k = k0 + kk, r = r0 + tx;
            float a = 0.f, b = 0.f;
            if (r < J.R && k < J.K) { a = J.re[(long long)k * J.ld + r]; b = J.im[(long long)k * J.ld + r]; }
            tre[tx][kk] = a; tim[tx][kk] = b;
        }
    }
    __syncthreads();
    const int R = J.R, K = J.K, ns = J.nsplit;
    const long long kp = J.kp;
    const int k = k0 + 2 * tx;
    if (k >= K) return;
    const bool two = (k + 1 < K);
    for (int i = ty; i < 32; i += 8) {
        int r = r0 + i;
        if (r >= R) break;
        __nv_bfloat16 a0[3], a1[3], b0[3], b1[3];
        split_bf16(tre[i][2 * tx], ns, a0);
        split_bf16(tim[i][2 * tx], ns, b0);
        split_bf16(two ? tre[i][2 * tx + 1] : 0.f, ns, a1);
        split_bf16(two ? tim[i][2 * tx + 1] : 0.f, ns, b1);
        #pragma unroll
        for (int p = 0; p < 3; ++p) {
            if (p >= ns) break;
            __nv_bfloat16 *o = J.out + p * J.plane_pitch;
            __nv_bfloat162 re2 = __halves2bfloat162(a0[p], a1[p]);
            __nv_bfloat162 im2 = __halves2bfloat162(b0[p], b1[p]);
            __nv_bfloat162 nim2 = __halves2bfloat162(__hneg(b0[p]), __hneg(b1[p]));
            auto st = [&](long long row, long long col, __nv_bfloat162 v) {
                if (two && ((row * kp + col) & 1) == 0) {
                    *reinterpret_cast<__nv_bfloat162 *>(o + row * kp + col) = v;
                } else {
                    o[row * kp + col] = v.x;
                    if (two) o[row * kp + col + 1] = v.y;
                }
            };
            if (!J.layoutB) {
                st(r, k, re2);
                st(r, K + k, im2);
            } else {
                st(r, k, re2);
                st(r, K + k, nim2);
                st(R + r, k, im2);
                st(R + r, K + k, re2);
            }
        }
    }
}

// Vectorised form of k_pack32 for whole 32 x 64 tiles (R % 32 == 0, K % 64 == 0,
// ld % 4 == 0, 16-byte aligned planes): 128-bit loads into shared memory, then
// each thread splits 8 consecutive k of one row and writes 16-byte rows of
// every plane.
__device__ __forceinline__ uint4 pack8(const __nv_bfloat16 (*v)[3], int p, bool neg) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat16 lo = v[2 * i][p], hi = v[2 * i + 1][p];
        if (neg) { lo = __hneg(lo); hi = __hneg(hi); }
        w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <int N>
__global__ void __launch_bounds__(256) k_pack32v(const __grid_constant__ PackJobsN<N> jobs) {
    const PackJob &J = jobs.j[blockIdx.z];
    __shared__ float tre[32][65], tim[32][65];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
    if (r0 >= J.R || k0 >= J.K) return;
    const int t = threadIdx.x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int idx = t + 256 * h;
        if (!J.trans) {
            const int row = idx >> 4, c4 = idx & 15;
            const long long g = (long long)(r0 + row) * J.ld + k0 + 4 * c4;
            const float4 a = *reinterpret_cast<const float4 *>(J.re + g), b = *reinterpret_cast<const float4 *>(J.im + g);
            tre[row][4 * c4] = a.x; tre[row][4 * c4 + 1] = a.y; tre[row][4 * c4 + 2] = a.z; tre[row][4 * c4 + 3] = a.w;
            tim[row][4 * c4] = b.x; tim[row][4 * c4 + 1] = b.y; tim[row][4 * c4 + 2] = b.z; tim[row][4 * c4 + 3] = b.w;
        } else {
            const int krow = idx >> 3, c4 = idx & 7;
            const long long g = (long long)(k0 + krow) * J.ld + r0 + 4 * c4;
            const float4 a = *reinterpret_cast<const float4 *>(J.re + g), b = *reinterpret_cast<const float4 *>(J.im + g);
            tre[4 * c4][krow] = a.x; tre[4 * c4 + 1][krow] = a.y; tre[4 * c4 + 2][krow] = a.z; tre[4 * c4 + 3][krow] = a.w;
            tim[4 * c4][krow] = b.x; tim[4 * c4 + 1][krow] = b.y; tim[4 * c4 + 2][krow] = b.z; tim[4 * c4 + 3][krow] = b.w;
        }
    }
    __syncthreads();
    const int r = t >> 3, c = t & 7;
    const int row = r0 + r, k = k0 + 8 * c;
    __nv_bfloat16 sr[8][3], si[8][3];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        split_bf16(tre[r][8 * c + u], J.nsplit, sr[u]);
        split_bf16(tim[r][8 * c + u], J.nsplit, si[u]);
    }
    const long long kp = J.kp, K = J.K, R = J.R;
    #pragma unroll
    for (int p = 0; p < 3; ++p) {
        if (p >= J.nsplit) break;
        __nv_bfloat16 *o = J.out + p * J.plane_pitch;
        const uint4 re = pack8(sr, p, false), im = pack8(si, p, false);
        if (!J.layoutB) {
            *reinterpret_cast<uint4 *>(o + row * kp + k) = re;
            *reinterpret_cast<uint4 *>(o + row * kp + K + k) = im;
        } else {
            *reinterpret_cast<uint4 *>(o + row * kp + k) = re;
            *reinterpret_cast<uint4 *>(o + row * kp + K + k) = pack8(si, p, true);
            *reinterpret_cast<uint4 *>(o + (R + row) * kp + k) = im;
            *reinterpret_cast<uint4 *>(o + (R + row) * kp + K + k) = re;
        }
    }
}

// A-layout pack of complex float64 rows (optionally the sum of two sources):
// row r = [Re v(r,:), Im v(r,:)], v = s1 (+ s2).
__global__ void k_pack64_A(const __grid_constant__ Tab<const double2 *> s1t, const __grid_constant__ Tab<const double2 *> s2t, long long ld, int R, int K,
                           int nsplit, const __grid_constant__ Tab<__nv_bfloat16 *> outt, long long kp, long long plane_pitch) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (k >= K || r >= R) return;
    const double2 *__restrict__ s1 = s1t.v[blockIdx.z], *__restrict__ s2 = s2t.v[blockIdx.z];
    __nv_bfloat16 *out = outt.v[blockIdx.z];
    double2 v = s1[(long long)r * ld + k];
    if (s2) v = cadd(v, s2[(long long)r * ld + k]);
    __nv_bfloat16 sa[3], sb[3];
    split_bf16((float)v.x, nsplit, sa);
    split_bf16((float)v.y, nsplit, sb);
    #pragma unroll
    for (int p = 0; p < 3; ++p) {
        if (p >= nsplit) break;
        __nv_bfloat16 *o = out + p * plane_pitch + (long long)r * kp;
        o[k] = sa[p];
        o[K + k] = sb[p];
    }
}

// B-layout pack of the transpose of complex float64 rows: logical
// v(r, k) = src[k][r] (r < R, k < K) -> rows r and R + r.
__global__ void k_pack64_BT(const __grid_constant__ Tab<const double2 *> srct, long long ld, int R, int K, int nsplit,
                            const __grid_constant__ Tab<__nv_bfloat16 *> outt, long long kp, long long plane_pitch) {
    __shared__ double2 t[32][33];
    const double2 *__restrict__ src = srct.v[blockIdx.z];
    __nv_bfloat16 *out = outt.v[blockIdx.z];
    int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += 8) {
        int k = k0 + i, r = r0 + tx;
        double2 v = cmk(0, 0);
        if (r < R && k < K) v = src[(long long)k * ld + r];
        t[tx][i] = v;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        int r = r0 + i, k = k0 + tx;
        if (r >= R || k >= K) continue;
        double2 v = t[i][tx];
        __nv_bfloat16 sa[3], sb[3];
        split_bf16((float)v.x, nsplit, sa);
        split_bf16((float)v.y, nsplit, sb);
        #pragma unroll
        for (int p = 0; p < 3; ++p) {
            if (p >= nsplit) break;
            __nv_bfloat16 *o = out + p * plane_pitch;
            o[(long long)r * kp + k] = sa[p];
            o[(long long)r * kp + K + k] = __hneg(sb[p]);
            o[(long long)(R + r) * kp + k] = sb[p];
            o[(long long)(R + r) * kp + K + k] = sa[p];
        }
    }
}

// X_j = K_j - G_{j-1} in float32 planes (K_j: 5-point slab block plus the
// boundary circulants on the first / last slab row).
// X_j = K_j - G_{j-1} in float32 planes (K_j: 4 - k^2 eps on the diagonal,
// -1 on the periodic neighbours, the circulants Sigma_bot / Sigma_top on the
// first / last slab row).  Thread: 4 consecutive columns xp of row x (n % 4 == 0).
__global__ void k_assemble32(GridDev g, int row, const __grid_constant__ Tab<const double *> epst, const double2 *circ,
                             const __grid_constant__ Tab<const float *> Gret, const __grid_constant__ Tab<const float *> Gimt, const __grid_constant__ Tab<float *> Xret, const __grid_constant__ Tab<float *> Ximt) {
    const int b = blockIdx.z;
    const double *eps = epst.v[b];
    const float *Gre = Gret.v[b], *Gim = Gimt.v[b];
    float *Xre = Xret.v[b], *Xim = Ximt.v[b];
    const int n = g.nx;
    const int x = blockIdx.y;
    const int xp0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (xp0 >= n) return;
    const long long idx = (long long)x * n + xp0;
    float vr[4] = {0.f, 0.f, 0.f, 0.f}, vi[4] = {0.f, 0.f, 0.f, 0.f};
    if (Gre) {
        const float4 a = *reinterpret_cast<const float4 *>(Gre + idx), b = *reinterpret_cast<const float4 *>(Gim + idx);
        vr[0] = -a.x; vr[1] = -a.y; vr[2] = -a.z; vr[3] = -a.w;
        vi[0] = -b.x; vi[1] = -b.y; vi[2] = -b.z; vi[3] = -b.w;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int xp = xp0 + u;
        float kr = 0.f, ki = 0.f;
        // float64 only on the one diagonal element (the FP64 pipe is narrow)
        if (xp == x) kr = (float)(4.0 - g.k * g.k * eps[(long long)row * n + x]);
        const int dx = x - xp;
        if (dx == 1 || dx == -1 || dx == n - 1 || dx == 1 - n) kr -= 1.f;
        if (n == 2 && dx != 0) kr -= 1.f;  // both periodic neighbours coincide
        const int d = dx < 0 ? dx + n : dx;
        if (row == 0) { kr += (float)circ[d].x; ki += (float)circ[d].y; }
        if (row == g.h - 1) { kr += (float)circ[n + d].x; ki += (float)circ[n + d].y; }
        vr[u] += kr;
        vi[u] += ki;
    }
    *reinterpret_cast<float4 *>(Xre + idx) = make_float4(vr[0], vr[1], vr[2], vr[3]);
    *reinterpret_cast<float4 *>(Xim + idx) = make_float4(vi[0], vi[1], vi[2], vi[3]);
}

// Symmetric random butterfly transform (depth 2) of an n x n complex-symmetric
// block in planar float32, in place.  U = P Q with Q the n-point butterfly
// (1/sqrt2)[R0 R1; R0 -R1] and P = diag of two n/2-point butterflies, R* random
// diagonals near 1; such a two-sided transform spreads every row over rows
// n/4 apart, so that the leading blocks of the Schur recursion (which pivots
// only inside its 32 x 32 leaves) are not the nearly singular sub-blocks of a
// strongly structured slab (high-contrast ridges) -- the randomisation that
// lets symmetric indefinite elimination run without pivoting.
//   forward: X' = U^T X U   (rows and columns: P^T then Q^T);
//   inverse: G  = U Y U^T   (rows and columns: Q then P).
// w[0 .. n): level-Q diagonals (R0 at i, R1 at n/2 + i); w[n .. 2n): level-P,
// half h (0 / 1) at n + h n/2 (R0 at i, R1 at n/4 + i).  One thread per 4 x 4
// group of rows {i, i+n/4, i+n/2, i+3n/4} x columns {j, ...}, i, j < n/4.
__device__ __forceinline__ void bf_fwd(float2 &t, float2 &b, float wa, float wb) {
    const float c = 0.70710678118654752f;
    const float2 s = make_float2(t.x + b.x, t.y + b.y), d = make_float2(t.x - b.x, t.y - b.y);
    t = make_float2(c * wa * s.x, c * wa * s.y);
    b = make_float2(c * wb * d.x, c * wb * d.y);
}
__device__ __forceinline__ void bf_inv(float2 &t, float2 &b, float wa, float wb) {
    const float c = 0.70710678118654752f;
    const float2 u = make_float2(wa * t.x, wa * t.y), v = make_float2(wb * b.x, wb * b.y);
    t = make_float2(c * (u.x + v.x), c * (u.y + v.y));
    b = make_float2(c * (u.x - v.x), c * (u.y - v.y));
}
template <bool INV>
__global__ void k_butterfly(const __grid_constant__ Tab<float *> ret, const __grid_constant__ Tab<float *> imt, long long ld, int n, const float *w) {
    float *re = ret.v[blockIdx.z], *im = imt.v[blockIdx.z];
    const int q = n >> 2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= q || i >= q) return;
    float2 m[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long g = (long long)(i + r * q) * ld + (j + c * q);
            m[r][c] = make_float2(re[g], im[g]);
        }
    // P level pairs (0,1) [half 0] and (2,3) [half 1] at local index i / j;
    // Q level pairs (0,2) and (1,3) at index i, i + q (resp. j, j + q)
    auto rows = [&](int a, int b, float wa, float wb) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (INV) bf_inv(m[a][c], m[b][c], wa, wb);
            else bf_fwd(m[a][c], m[b][c], wa, wb);
        }
    };
    auto cols = [&](int a, int b, float wa, float wb) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (INV) bf_inv(m[r][a], m[r][b], wa, wb);
            else bf_fwd(m[r][a], m[r][b], wa, wb);
        }
    };
    const float *wq = w, *wp0 = w + n, *wp1 = w + n + n / 2;
    if (!INV) {
        rows(0, 1, wp0[i], wp0[q + i]); rows(2, 3, wp1[i], wp1[q + i]);
        rows(0, 2, wq[i], wq[2 * q + i]); rows(1, 3, wq[q + i], wq[3 * q + i]);
        cols(0, 1, wp0[j], wp0[q + j]); cols(2, 3, wp1[j], wp1[q + j]);
        cols(0, 2, wq[j], wq[2 * q + j]); cols(1, 3, wq[q + j], wq[3 * q + j]);
    } else {
        rows(0, 2, wq[i], wq[2 * q + i]); rows(1, 3, wq[q + i], wq[3 * q + i]);
        rows(0, 1, wp0[i], wp0[q + i]); rows(2, 3, wp1[i], wp1[q + i]);
        cols(0, 2, wq[j], wq[2 * q + j]); cols(1, 3, wq[q + j], wq[3 * q + j]);
        cols(0, 1, wp0[j], wp0[q + j]); cols(2, 3, wp1[j], wp1[q + j]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long g = (long long)(i + r * q) * ld + (j + c * q);
            re[g] = m[r][c].x;
            im[g] = m[r][c].y;
        }
}

// Float32 Gauss-Jordan inverse of an n x n (n <= 128) diagonal block with
// partial pivoting, in shared memory (planar in global memory).
__global__ void __launch_bounds__(512) k_leaf_inv32(float *re, float *im, long long ld, int n, int *flags) {
    extern __shared__ float2 a32[];
    __shared__ float2 colk[128];
    __shared__ int piv[128];
    __shared__ int s_p;
    __shared__ float2 s_inv;
    int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) {
        long long gidx = (long long)(e / n) * ld + (e % n);
        a32[e] = make_float2(re[gidx], im[gidx]);
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            float best = -1.f;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                float2 v = a32[i * n + k];
                float m = v.x * v.x + v.y * v.y;
                if (m > best) { best = m; bi = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                float ob = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                s_p = bi;
                piv[k] = bi;
                if (!(best > 0.f) || !isfinite(best)) atomicOr(flags, FLAG_SINGULAR);
            }
        }
        __syncthreads();
        int p = s_p;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                float2 t = a32[k * n + j];
                a32[k * n + j] = a32[p * n + j];
                a32[p * n + j] = t;
            }
            __syncthreads();
        }
        if (tid == 0) {
            float2 d = a32[k * n + k];
            float den = d.x * d.x + d.y * d.y;
            s_inv = make_float2(d.x / den, -d.y / den);
        }
        __syncthreads();
        float2 inv = s_inv;
        for (int j = tid; j < n; j += nt) a32[k * n + j] = (j == k) ? inv : fmul(a32[k * n + j], inv);
        for (int i = tid; i < n; i += nt) colk[i] = a32[i * n + k];
        __syncthreads();
        for (int e = tid; e < n * n; e += nt) {
            int i = e / n, j = e - i * n;
            if (i == k) continue;
            float2 f = colk[i];
            if (j == k) {
                float2 t = fmul(f, inv);
                a32[e] = make_float2(-t.x, -t.y);
            } else {
                float2 t = fmul(f, a32[k * n + j]);
                a32[e] = make_float2(a32[e].x - t.x, a32[e].y - t.y);
            }
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k) {
            for (int i = tid; i < n; i += nt) {
                float2 t = a32[i * n + k];
                a32[i * n + k] = a32[i * n + p];
                a32[i * n + p] = t;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt) {
        long long gidx = (long long)(e / n) * ld + (e % n);
        re[gidx] = a32[e].x;
        im[gidx] = a32[e].y;
    }
}

template <int NB>
__global__ void __launch_bounds__(NB * 4) k_leaf32(float *re, float *im, long long ld, int *flags) {
    LeafIO<float, true> io{re, im, nullptr, ld};
    leaf_gj<float, NB, true>(io, flags);
}

template <int NB>
__global__ void __launch_bounds__(NB * 4) k_leaf32r(float *re, float *im, long long ld, int *flags) {
    leaf_gj_regs<NB>(re, im, ld, flags);
}

__global__ void __launch_bounds__(512) k_leaf128rec(const __grid_constant__ Tab<float *> re, const __grid_constant__ Tab<float *> im, long long ld, const __grid_constant__ Tab<int *> flags) {
    const int b = blockIdx.x;
    leaf128_recursive(re.v[b], im.v[b], ld, flags.v[b]);
}

template <int NB>
__global__ void __launch_bounds__(NB * 4) k_leaf32r2(float *re, float *im, long long ld, int *flags) {
    leaf_gj_regs2<NB>(re, im, ld, flags);
}

// C block <- -V, B block <- -V^T (planar float32).
__global__ void k_negoff32(const __grid_constant__ Tab<float *> Bret, const __grid_constant__ Tab<float *> Bimt, const __grid_constant__ Tab<float *> Cret, const __grid_constant__ Tab<float *> Cimt, long long ld,
                           const __grid_constant__ Tab<const float *> Vret, const __grid_constant__ Tab<const float *> Vimt, int h) {
    __shared__ float tr[32][33], ti[32][33];
    const int b = blockIdx.z;
    float *Bre = Bret.v[b], *Bim = Bimt.v[b], *Cre = Cret.v[b], *Cim = Cimt.v[b];
    const float *Vre = Vret.v[b], *Vim = Vimt.v[b];
    int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += 8) {
        int gi = i0 + i, gj = j0 + tx;
        if (gi < h && gj < h) {
            float vr = Vre[(long long)gi * h + gj], vi = Vim[(long long)gi * h + gj];
            Cre[(long long)gi * ld + gj] = -vr;
            Cim[(long long)gi * ld + gj] = -vi;
            tr[i][tx] = vr; ti[i][tx] = vi;
        }
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        int gj = j0 + i, gi = i0 + tx;  // B[gj][gi] = -V[gi][gj]
        if (gi < h && gj < h) {
            Bre[(long long)gj * ld + gi] = -tr[tx][i];
            Bim[(long long)gj * ld + gi] = -ti[tx][i];
        }
    }
}

// E[c][x] = (R ? R[c][x] : 0) + O[c][x] for c < mcols;  E = R for c >= mcols.
__global__ void k_combine(const __grid_constant__ Tab<double2 *> Et, const __grid_constant__ Tab<const double2 *> Rt, const __grid_constant__ Tab<const float *> Oret,
                          const __grid_constant__ Tab<const float *> Oimt, int ncol, int mcols, int nx) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (x >= nx) return;
    const int b = blockIdx.z;
    double2 *E = Et.v[b];
    const double2 *R = Rt.v[b];
    const float *Ore = Oret.v[b], *Oim = Oimt.v[b];
    long long i = (long long)c * nx + x;
    double2 v = R ? R[i] : cmk(0, 0);
    if (c < mcols) { v.x += (double)Ore[i]; v.y += (double)Oim[i]; }
    E[i] = v;
    (void)ncol;
}

// out = Sigma in, Sigma = U diag(sigma) U^H (a circulant), per column:
// inverse DFT of sigma times the DFT of the column.
__global__ void k_circ_apply(const double2 *in, double2 *out, int n, int logn, const double2 *sigma,
                             const double2 *tw) {
    extern __shared__ double2 a[];
    const double2 *src = in + (long long)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[__brev((unsigned)i) >> (32 - logn)] = src[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int lh = 0; lh < logn; ++lh) {
            int half = 1 << lh, tstride = n >> (lh + 1);
            for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
                int pos = t & (half - 1);
                int i = ((t >> lh) << (lh + 1)) + pos, j = i + half;
                double2 w = tw[pos * tstride];
                if (pass == 1) w.y = -w.y;
                double2 u = a[i], v = cmul(a[j], w);
                a[i] = cadd(u, v);
                a[j] = csub(u, v);
            }
            __syncthreads();
        }
        if (pass == 0) {
            // multiply by sigma[m] and bit-reverse for the inverse transform
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                unsigned r = __brev((unsigned)i) >> (32 - logn);
                if ((int)r > i) {
                    double2 x = cmul(a[i], sigma[i]), y = cmul(a[r], sigma[r]);
                    a[i] = y;
                    a[r] = x;
                } else if ((int)r == i) {
                    a[i] = cmul(a[i], sigma[i]);
                }
            }
            __syncthreads();
        }
    }
    double2 *dst = out + (long long)blockIdx.x * n;
    double s = 1.0 / n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = cscale(a[i], s);
}

// r_j = R_j - K E restricted to the slab, float64.  K E at a pixel is
// d E - (sum of the four neighbours) + boundary terms, d = 4 - k^2 eps; the
// neighbour sum and the boundary terms are gathered first so that the
// diagonal term is one fused multiply-add per component.
__global__ void k_residual(GridDev g, const double *eps, const double2 *E, const double2 *R, const double2 *cb,
                           const double2 *ct, double2 *r, int ncol) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y, j = blockIdx.z;
    const int n = g.nx;
    if (x >= n) return;
    const long long L = (long long)ncol * n;
    const double2 *e = E + j * L + (long long)c * n;
    const double d = fma(-(g.k * g.k), eps[(long long)j * n + x], 4.0);
    const int xr = (x + 1 == n) ? 0 : x + 1, xl = (x == 0) ? n - 1 : x - 1;
    double2 nbr = cadd(e[xr], e[xl]);  // neighbours minus boundary terms
    if (j > 0) nbr = cadd(nbr, e[x - L]);
    if (j < g.h - 1) nbr = cadd(nbr, e[x + L]);
    if (j == 0) nbr = csub(nbr, cb[(long long)c * n + x]);
    if (j == g.h - 1) nbr = csub(nbr, ct[(long long)c * n + x]);
    const double2 ex = e[x];
    const double2 v = make_double2(fma(d, ex.x, -nbr.x), fma(d, ex.y, -nbr.y));
    const long long idx = j * L + (long long)c * n + x;
    r[idx] = R ? csub(R[idx], v) : v;  // without R: K E
}

// out[c] = sum_{j,x} |X_j[c][x]|^2 (one block of 256 threads per column, a
// fixed summation order; two independent loads in flight per thread).  With
// `copy`, X is also copied there.
__global__ void __launch_bounds__(256) k_colnorm(const double2 *X, int h, int ncol, int nx, double *out,
                                                 double2 *copy) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    double a0 = 0.0, a1 = 0.0;
    for (int j = 0; j < h; ++j) {
        const long long o = ((long long)j * ncol + c) * nx;
        const double2 *p = X + o;
        int x = threadIdx.x;
        for (; x + 256 < nx; x += 512) {
            const double2 u = p[x], v = p[x + 256];
            if (copy) {
                copy[o + x] = u;
                copy[o + x + 256] = v;
            }
            a0 += cabs2(u);
            a1 += cabs2(v);
        }
        if (x < nx) {
            const double2 u = p[x];
            if (copy) copy[o + x] = u;
            a0 += cabs2(u);
        }
    }
    red[threadIdx.x] = a0 + a1;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// Krylov helpers over fields [row][column][x]: per-column dot products
// (conj(A) . B, one block per column, fixed order), Y += sgn coef[c] X, and
// Y = X / sqrt(nrm2[c]) (zero when the norm is zero).
__global__ void k_coldot(const double2 *A, const double2 *B, int h, int ncol, int nx, double2 *out) {
    __shared__ double2 red[256];
    const int c = blockIdx.x;
    double2 acc = cmk(0.0, 0.0);
    for (int j = 0; j < h; ++j) {
        const long long o = ((long long)j * ncol + c) * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) acc = cadd(acc, cmul(cconj(A[o + x]), B[o + x]));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

__global__ void k_colaxpy(double2 *Y, const double2 *X, const double2 *coef, double sgn, int ncol, int nx) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y, j = blockIdx.z;
    if (x >= nx) return;
    const long long i = ((long long)j * ncol + c) * nx + x;
    Y[i] = cadd(Y[i], cscale(cmul(coef[c], X[i]), sgn));
}

__global__ void k_colscale(double2 *Y, const double2 *X, const double *nrm2, int ncol, int nx) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y, j = blockIdx.z;
    if (x >= nx) return;
    const long long i = ((long long)j * ncol + c) * nx + x;
    const double n2 = nrm2[c];
    Y[i] = n2 > 0.0 ? cscale(X[i], 1.0 / sqrt(n2)) : cmk(0.0, 0.0);
}

__global__ void k_axpy(double2 *E, const double2 *d, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) E[i] = cadd(E[i], d[i]);
}

// g_j(x) = 2 k^2 Re sum_b Phi_j[b][x] Q[b][x].  Block: 32 consecutive x (lanes)
// x 8 warps, warp w summing b = w, w + 8, ...; the 8 partial sums are added in
// a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_grad_rowdot32(const __grid_constant__ Tab<const double2 *> Et, const __grid_constant__ Tab<const float *> Qret,
                                                       const __grid_constant__ Tab<const float *> Qimt, int j, int nx, int n_in, int n_out,
                                                       double k2, const __grid_constant__ Tab<double *> gt) {
    __shared__ double part[8][32];
    const double2 *E = Et.v[blockIdx.z];
    const float *Qre = Qret.v[blockIdx.z], *Qim = Qimt.v[blockIdx.z];
    double *g = gt.v[blockIdx.z];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int ncol = n_in + n_out;
    double acc = 0.0;
    if (x < nx) {
        const double2 *phi = E + ((long long)j * ncol + n_in) * nx + x;
        for (int b = w; b < n_out; b += 8) {
            const double2 p = phi[(long long)b * nx];
            acc = fma(p.x, (double)Qre[(long long)b * nx + x], acc);
            acc = fma(-p.y, (double)Qim[(long long)b * nx + x], acc);
        }
    }
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && x < nx) {
        double t = part[0][lane];
#pragma unroll
        for (int i = 1; i < 8; ++i) t += part[i][lane];
        g[(long long)j * nx + x] = 2.0 * k2 * t;
    }
}

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

template <typename T>
int walloc(apf_ctx *c, MixedWork *w, T **p, long long count) {
    void *q = nullptr;
    size_t bytes = (size_t)std::max<long long>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, APF_ENOMEM, "cudaMalloc(%zu) for the mixed workspace failed", bytes);
    }
    w->allocs.push_back(q);
    c->ws_bytes += (long long)bytes;
    *p = (T *)q;
    return APF_OK;
}

// ---- host-side helpers ----------------------------------------------------
struct PV {  // planar complex view
    float *re, *im;
    long long ld;
    PV off(long long r, long long c) const { return PV{re + r * ld + c, im + r * ld + c, ld}; }
};

PackJob make_job(__nv_bfloat16 *dst, const PV &src, int R, int K, bool trans, bool layoutB, int nsplit,
                 PackView *view) {
    long long kp = round_up(2LL * K, 64);
    long long rows = layoutB ? 2LL * R : R;
    *view = PackView{dst, rows, kp, nsplit, rows * kp};
    return PackJob{src.re, src.im, src.ld, R, K, trans ? 1 : 0, layoutB ? 1 : 0, nsplit, dst, kp, rows * kp};
}

template <int N>
void launch_jobs_n(apf_ctx *c, const PackJob *js, int nj, cudaStream_t s) {
    PackJobsN<N> jobs{};
    int maxR = 0, maxK = 0;
    for (int i = 0; i < nj; ++i) {
        jobs.j[i] = js[i];
        if (js[i].kp != 2LL * js[i].K)
            cudaMemsetAsync(js[i].out, 0, sizeof(__nv_bfloat16) * (js[i].plane_pitch * js[i].nsplit), s);
        maxR = std::max(maxR, js[i].R);
        maxK = std::max(maxK, js[i].K);
    }
    dim3 grid((maxK + 63) / 64, (maxR + 31) / 32, nj);
    bool vec = true;
    for (int i = 0; i < nj; ++i) {
        const PackJob &J = js[i];
        vec = vec && J.R % 32 == 0 && J.K % 64 == 0 && J.ld % 4 == 0 && J.R == maxR && J.K == maxK &&
              ((((uintptr_t)J.re) | ((uintptr_t)J.im) | ((uintptr_t)J.out)) & 15) == 0 && J.kp % 8 == 0 &&
              J.plane_pitch % 8 == 0;
    }
    if (vec) APF_LAUNCH(c, k_pack32v<N>, grid, 256, 0, s, jobs);
    else APF_LAUNCH(c, k_pack32<N>, grid, dim3(32, 8), 0, s, jobs);
}

void launch_jobs(apf_ctx *c, const PackJob *js, int nj, cudaStream_t s) {
    if (nj <= 2) launch_jobs_n<2>(c, js, nj, s);
    else launch_jobs_n<MAX_JOBS>(c, js, nj, s);
}

PackView pack32(apf_ctx *c, __nv_bfloat16 *dst, const PV &src, int R, int K, bool trans, bool layoutB, int nsplit,
                cudaStream_t s) {
    PackView v;
    PackJob j = make_job(dst, src, R, K, trans, layoutB, nsplit, &v);
    launch_jobs(c, &j, 1, s);
    return v;
}

// The designs of one call: every step below launches once for all of them
// (they share grid, slab height, channel set and settings; each has its own
// buffers).  A single design is a batch of one.
struct Bat {
    int n = 1;
    apf_ctx *c[TC_MAX_BATCH] = {};
    apf_ctx *lead() const { return c[0]; }
};

Bat one(apf_ctx *c) {
    Bat b;
    b.n = 1;
    b.c[0] = c;
    return b;
}

template <typename T, typename F>
Tab<T> tab(const Bat &bt, F f) {
    Tab<T> t{};
    for (int b = 0; b < bt.n; ++b) t.v[b] = f(b);
    return t;
}

// Pack the A operand sa[b] and the B operand sb[b] of one product for every
// design (in w->PA / w->PB of each design) in one launch.
void pack2_b(const Bat &bt, PackView *va, const PV *sa, int Ra, int Ka, bool ta, PackView *vb, const PV *sb, int Rb,
             int Kb, bool tb, int nsplit, cudaStream_t s) {
    PackJob js[2 * TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) {
        MixedWork *w = bt.c[b]->mw;
        js[2 * b] = make_job(w->PA, sa[b], Ra, Ka, ta, false, nsplit, &va[b]);
        js[2 * b + 1] = make_job(w->PB, sb[b], Rb, Kb, tb, true, nsplit, &vb[b]);
    }
    launch_jobs(bt.lead(), js, 2 * bt.n, s);
}

void pack32_b(const Bat &bt, PackView *v, __nv_bfloat16 *const *dst, const PV *src, int R, int K, bool trans,
              bool layoutB, int nsplit, cudaStream_t s) {
    PackJob js[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) js[b] = make_job(dst[b], src[b], R, K, trans, layoutB, nsplit, &v[b]);
    launch_jobs(bt.lead(), js, bt.n, s);
}

void pack64A_b(const Bat &bt, PackView *v, __nv_bfloat16 *const *dst, const double2 *const *s1,
               const double2 *const *s2, long long ld, int R, int K, int nsplit, cudaStream_t s) {
    const long long kp = round_up(2LL * K, 64);
    for (int b = 0; b < bt.n; ++b) {
        if (kp != 2LL * K) cudaMemsetAsync(dst[b], 0, sizeof(__nv_bfloat16) * R * kp * nsplit, s);
        v[b] = PackView{dst[b], R, kp, nsplit, (long long)R * kp};
    }
    dim3 grid((K + 255) / 256, R, bt.n);
    APF_LAUNCH(bt.lead(), k_pack64_A, grid, 256, 0, s, tab<const double2 *>(bt, [&](int b) { return s1[b]; }),
               tab<const double2 *>(bt, [&](int b) { return s2 ? s2[b] : nullptr; }), ld, R, K, nsplit,
               tab<__nv_bfloat16 *>(bt, [&](int b) { return dst[b]; }), kp, (long long)R * kp);
}

void pack64BT_b(const Bat &bt, PackView *v, __nv_bfloat16 *const *dst, const double2 *const *src, long long ld, int R,
                int K, int nsplit, cudaStream_t s) {
    const long long kp = round_up(2LL * K, 64);
    const long long rows = 2LL * R;
    for (int b = 0; b < bt.n; ++b) {
        if (kp != 2LL * K) cudaMemsetAsync(dst[b], 0, sizeof(__nv_bfloat16) * rows * kp * nsplit, s);
        v[b] = PackView{dst[b], rows, kp, nsplit, rows * kp};
    }
    dim3 grid((K + 31) / 32, (R + 31) / 32, bt.n);
    APF_LAUNCH(bt.lead(), k_pack64_BT, grid, dim3(32, 8), 0, s,
               tab<const double2 *>(bt, [&](int b) { return src[b]; }), ld, R, K, nsplit,
               tab<__nv_bfloat16 *>(bt, [&](int b) { return dst[b]; }), kp, rows * kp);
}

// out[b] = alpha A[b] B[b]^T + beta in[b] for every design, one launch.
int gemm_b(const Bat &bt, const PackView *A, const PackView *B, int nsplit, int M, int N, int n_cplx, float alpha,
           float beta, const PV *out, const PV *in, cudaStream_t s) {
    TcProblem pb[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b)
        pb[b] = TcProblem{A[b], B[b], out[b].re, out[b].im, in ? in[b].re : nullptr, in ? in[b].im : nullptr,
                          bt.c[b]->d_flags};
    return tc_gemm_n(bt.lead(), bt.n, pb, nsplit, M, N, n_cplx, alpha, beta, out[0].ld, in ? in[0].ld : 0, s);
}

int leaf_size(const MixedWork *w) { return w->leaf; }

// Diagonal block of the recursion, one design (kernel variant per the context's knobs).
void leaf_one(apf_ctx *lead, const PV &X, int n, int *flags, cudaStream_t s) {
    MixedWork *w = lead->mw;
    Tab<float *> re{}, im{};
    Tab<int *> fl{};
    re.v[0] = X.re; im.v[0] = X.im; fl.v[0] = flags;
    // 128 blocks: in-CTA Schur recursion over 32 x 32 Gauss-Jordan leaves
    // (default); variants 1-3 are the single-level Gauss-Jordan kernels.
    if (n == 128 && w->leaf_variant == 1)
        APF_LAUNCH(lead, k_leaf32r2<128>, 1, 512, 0, s, X.re, X.im, X.ld, flags);
    else if (n == 128 && w->leaf_variant == 2)
        APF_LAUNCH(lead, k_leaf32<128>, 1, 512, leaf_smem_bytes<128>(8), s, X.re, X.im, X.ld, flags);
    else if (n == 128 && w->leaf_variant == 3)
        APF_LAUNCH(lead, k_leaf32r<128>, 1, 512, 0, s, X.re, X.im, X.ld, flags);
    else if (n == 128)
        APF_LAUNCH(lead, k_leaf128rec, 1, 512, rec_smem_bytes(), s, re, im, X.ld, fl);
    else if (n == 64 && w->leaf_variant == 1)
        APF_LAUNCH(lead, k_leaf32r2<64>, 1, 256, 0, s, X.re, X.im, X.ld, flags);
    else if (n == 64)
        APF_LAUNCH(lead, k_leaf32r<64>, 1, 256, 0, s, X.re, X.im, X.ld, flags);
    else if (n == 32)
        APF_LAUNCH(lead, k_leaf32<32>, 1, 128, leaf_smem_bytes<32>(8), s, X.re, X.im, X.ld, flags);
    else if (n == 16)
        APF_LAUNCH(lead, k_leaf32<16>, 1, 64, leaf_smem_bytes<16>(8), s, X.re, X.im, X.ld, flags);
    else
        APF_LAUNCH(lead, k_leaf_inv32, 1, 256, n * n * (int)sizeof(float2), s, X.re, X.im, X.ld, n, flags);
}

// X[b] <- X[b]^-1 in place for complex-symmetric X[b], every design of the
// batch: the 2x2 block Schur recursion of the float64 path with all four
// products on the tensor cores.
int inv32_b(const Bat &bt, const PV *X, int n, float *const *Tre, float *const *Tim, float *const *Vre,
            float *const *Vim, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    MixedWork *w = c->mw;
    const int nb = bt.n;
    if (n <= leaf_size(w)) {
        if (n == 128 && w->leaf_variant == 0) {
            // one CTA per design's block
            APF_LAUNCH(c, k_leaf128rec, nb, 512, rec_smem_bytes(), s, tab<float *>(bt, [&](int b) { return X[b].re; }),
                       tab<float *>(bt, [&](int b) { return X[b].im; }), X[0].ld,
                       tab<int *>(bt, [&](int b) { return bt.c[b]->d_flags; }));
        } else {
            for (int b = 0; b < nb; ++b) leaf_one(c, X[b], n, bt.c[b]->d_flags, s);
        }
        return APF_OK;
    }
    const int h = n / 2;
    const int ns = w->nsplit_elim;
    const long long hh = (long long)h * h;
    PV A[TC_MAX_BATCH], B[TC_MAX_BATCH], C[TC_MAX_BATCH], D[TC_MAX_BATCH], T[TC_MAX_BATCH], V[TC_MAX_BATCH];
    float *tr2[TC_MAX_BATCH], *ti2[TC_MAX_BATCH], *vr2[TC_MAX_BATCH], *vi2[TC_MAX_BATCH];
    for (int b = 0; b < nb; ++b) {
        A[b] = X[b]; B[b] = X[b].off(0, h); C[b] = X[b].off(h, 0); D[b] = X[b].off(h, h);
        T[b] = PV{Tre[b], Tim[b], h}; V[b] = PV{Vre[b], Vim[b], h};
        tr2[b] = Tre[b] + hh; ti2[b] = Tim[b] + hh; vr2[b] = Vre[b] + hh; vi2[b] = Vim[b] + hh;
    }
    int rc;
    PackView pa[TC_MAX_BATCH], pb[TC_MAX_BATCH];
    if ((rc = inv32_b(bt, A, h, tr2, ti2, vr2, vi2, s))) return rc;
    // T = C Ai
    pack2_b(bt, pa, C, h, h, false, pb, A, h, h, false, ns, s);
    if ((rc = gemm_b(bt, pa, pb, ns, h, 2 * h, h, 1.f, 0.f, T, nullptr, s))) return rc;
    // D = D - T B   (B-operand columns = rows of C)
    pack2_b(bt, pa, T, h, h, false, pb, C, h, h, false, ns, s);
    if ((rc = gemm_b(bt, pa, pb, ns, h, 2 * h, h, -1.f, 1.f, D, D, s))) return rc;
    if ((rc = inv32_b(bt, D, h, tr2, ti2, vr2, vi2, s))) return rc;
    // V = Si T
    pack2_b(bt, pa, D, h, h, false, pb, T, h, h, true, ns, s);
    if ((rc = gemm_b(bt, pa, pb, ns, h, 2 * h, h, 1.f, 0.f, V, nullptr, s))) return rc;
    // A = Ai + V^T T   (the B operand is still the packed T^T)
    __nv_bfloat16 *padst[TC_MAX_BATCH];
    for (int b = 0; b < nb; ++b) padst[b] = bt.c[b]->mw->PA;
    pack32_b(bt, pa, padst, V, h, h, true, false, ns, s);
    if ((rc = gemm_b(bt, pa, pb, ns, h, 2 * h, h, 1.f, 1.f, A, A, s))) return rc;
    dim3 grid((h + 31) / 32, (h + 31) / 32, nb);
    APF_LAUNCH(c, k_negoff32, grid, dim3(32, 8), 0, s, tab<float *>(bt, [&](int b) { return B[b].re; }),
               tab<float *>(bt, [&](int b) { return B[b].im; }), tab<float *>(bt, [&](int b) { return C[b].re; }),
               tab<float *>(bt, [&](int b) { return C[b].im; }), X[0].ld,
               tab<const float *>(bt, [&](int b) { return (const float *)V[b].re; }),
               tab<const float *>(bt, [&](int b) { return (const float *)V[b].im; }), h);
    return APF_OK;
}

int inv32(apf_ctx *c, const PV &X, int n, float *Tre, float *Tim, float *Vre, float *Vim, cudaStream_t s) {
    return inv32_b(one(c), &X, n, &Tre, &Tim, &Vre, &Vim, s);
}

// Packed operand view of G_j (slot j, or j's slot in its segment).
PackView gp_view(const apf_ctx *c, int j) {
    const MixedWork *w = c->mw;
    const long long rows = 2LL * c->nx, kp = 2LL * c->nx;
    const int slot = w->seg_rows > 0 ? j % w->seg_rows : j;
    return PackView{w->GP + slot * w->gp_stride, rows, kp, w->nsplit_elim, rows * kp};
}

// E[b] ~= Khat[b]^-1 Rin[b] with the stored (or recomputed) G_j of each design
// (block forward sweep + back substitution).  mcols: columns that the forward
// sweep must carry.
int approx_solve_b(const Bat &bt, const double2 *const *Rin, double2 *const *Eout, int mcols, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    MixedWork *w = c->mw;
    const int nb = bt.n;
    const int ncol = c->cf + c->ca;
    const int nx = c->nx, ns = w->nsplit_elim;
    const long long L = (long long)ncol * nx;
    const int K = w->seg_rows;
    // with recomputation: the segment whose inverses row j needs must be loaded
    auto need = [&](int j) -> int {
        if (K <= 0) return APF_OK;
        const int sg = j / K;
        if (sg == w->seg_loaded) return APF_OK;
        return recompute_segment_b(bt, sg, s);
    };
    PV O[TC_MAX_BATCH];
    __nv_bfloat16 *padst[TC_MAX_BATCH];
    for (int b = 0; b < nb; ++b) {
        MixedWork *wb = bt.c[b]->mw;
        O[b] = PV{wb->O32, wb->O32 + L, nx};
        padst[b] = wb->PA;
        cudaMemcpyAsync(Eout[b], Rin[b], sizeof(double2) * L, cudaMemcpyDeviceToDevice, s);
    }
    auto otab_re = tab<const float *>(bt, [&](int b) { return (const float *)O[b].re; });
    auto otab_im = tab<const float *>(bt, [&](int b) { return (const float *)O[b].im; });
    dim3 cgrid((nx + 255) / 256, ncol, nb);
    PackView pa[TC_MAX_BATCH], gv[TC_MAX_BATCH];
    const double2 *src[TC_MAX_BATCH], *src2[TC_MAX_BATCH];
    int rc;
    for (int j = 1; j < c->h; ++j) {
        if (mcols > 0) {
            if ((rc = need(j - 1))) return rc;
            for (int b = 0; b < nb; ++b) {
                src[b] = Eout[b] + (j - 1) * L;
                gv[b] = gp_view(bt.c[b], j - 1);
            }
            pack64A_b(bt, pa, padst, src, nullptr, nx, mcols, nx, ns, s);
            if ((rc = gemm_b(bt, pa, gv, ns, mcols, 2 * nx, nx, 1.f, 0.f, O, nullptr, s))) return rc;
        }
        APF_LAUNCH(c, k_combine, cgrid, 256, 0, s, tab<double2 *>(bt, [&](int b) { return Eout[b] + j * L; }),
                   tab<const double2 *>(bt, [&](int b) { return Rin[b] + j * L; }), otab_re, otab_im, ncol, mcols,
                   nx);
    }
    for (int j = c->h - 1; j >= 0; --j) {
        if ((rc = need(j))) return rc;
        for (int b = 0; b < nb; ++b) {
            src[b] = Eout[b] + j * L;
            src2[b] = (j == c->h - 1) ? nullptr : Eout[b] + (j + 1) * L;
            gv[b] = gp_view(bt.c[b], j);
        }
        pack64A_b(bt, pa, padst, src, (j == c->h - 1) ? nullptr : src2, nx, ncol, nx, ns, s);
        if ((rc = gemm_b(bt, pa, gv, ns, ncol, 2 * nx, nx, 1.f, 0.f, O, nullptr, s))) return rc;
        APF_LAUNCH(c, k_combine, cgrid, 256, 0, s, tab<double2 *>(bt, [&](int b) { return Eout[b] + j * L; }),
                   tab<const double2 *>(bt, [&](int b) { return (const double2 *)nullptr; }), otab_re, otab_im,
                   ncol, ncol, nx);
    }
    return APF_OK;
}

int approx_solve(apf_ctx *c, const double2 *Rin, double2 *Eout, int mcols, cudaStream_t s) {
    return approx_solve_b(one(c), &Rin, &Eout, mcols, s);
}

int residual(apf_ctx *c, const double2 *E, double2 *r, cudaStream_t s) {
    MixedWork *w = c->mw;
    int ncol = c->cf + c->ca;
    int nx = c->nx;
    long long L = (long long)ncol * nx;
    int logn = 0;
    while ((1 << logn) < nx) ++logn;
    int threads = nx / 2 < 256 ? nx / 2 : 256;
    int smem = nx * (int)sizeof(double2);
    APF_LAUNCH(c, k_circ_apply, ncol, threads, smem, s, E, w->cb, nx, logn, c->d_modes, c->d_tw);
    APF_LAUNCH(c, k_circ_apply, ncol, threads, smem, s, E + (c->h - 1) * L, w->ct, nx, logn, c->d_modes + nx,
               c->d_tw);
    GridDev g = make_grid(c);
    dim3 grid((nx + 255) / 256, ncol, c->h);
    APF_LAUNCH(c, k_residual, grid, 256, 0, s, g, c->d_eps, E, c->d_R, w->cb, w->ct, r, ncol);
    return APF_OK;
}

}  // namespace

void mixed_init_attrs() {
    tc_init_attrs();
    cudaFuncSetAttribute(k_leaf_inv32, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * (int)sizeof(float2));
    cudaFuncSetAttribute(k_leaf32<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem_bytes<128>(8));
    cudaFuncSetAttribute(k_leaf32<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem_bytes<64>(8));
    cudaFuncSetAttribute(k_leaf128rec, cudaFuncAttributeMaxDynamicSharedMemorySize, rec_smem_bytes());
    cudaFuncSetAttribute(k_circ_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * (int)sizeof(double2));
}

void mixed_free(apf_ctx *c) {
    if (!c->mw) return;
    for (void *p : c->mw->allocs) cudaFree(p);
    delete c->mw;
    c->mw = nullptr;
}

int mixed_alloc(apf_ctx *c) {
    mixed_free(c);
    MixedWork *w = new MixedWork();
    c->mw = w;
    w->nsplit_elim = c->elim_planes;
    if (const char *e = getenv("APF_NSPLIT_ELIM")) {  // tuning knob: bf16 planes of the elimination (2 or 3)
        int v = atoi(e);
        if (v == 2 || v == 3) w->nsplit_elim = v;
    }
    if (const char *e = getenv("APF_LEAF_VARIANT")) {  // tuning knob: 128-block leaf kernel (0..3)
        int v = atoi(e);
        if (v >= 0 && v <= 3) w->leaf_variant = v;
    }
    long long n = c->nx, h = c->h;
    int nin = c->nin, nout = c->nout;
    long long ncol = nin + nout;
    int rc;
#define WA(p, cnt) if ((rc = walloc(c, w, &(p), (cnt))) != APF_OK) return rc;
    WA(w->Xre, n * n); WA(w->Xim, n * n);
    WA(w->Tre, n * n / 2); WA(w->Tim, n * n / 2); WA(w->Vre, n * n / 2); WA(w->Vim, n * n / 2);
    int ns_max = std::max(w->nsplit_elim, w->nsplit_grad);
    // A operands: recursion (h x 2h), fields (ncol x 2n), Gamma (n_out x kp)
    long long kp_g = round_up(2LL * nin, 64);
    w->pa_elems = std::max({(n / 2) * n * w->nsplit_elim, ncol * 2 * n * w->nsplit_elim, (long long)nout * kp_g * ns_max});
    // B operands: recursion (2h x 2h), gradient (2n x kp_g)
    w->pb_elems = std::max(n * n * w->nsplit_elim, 2 * n * kp_g * ns_max);
    WA(w->PA, w->pa_elems);
    WA(w->PB, w->pb_elems);
    if (const char *e = getenv("APF_BUTTERFLY")) w->bfly = (e[0] == '1');  // diagnostic knob; default from ctx
    else w->bfly = c->butterfly;
    WA(w->BW, 2 * n);
    {
        // random diagonals exp(rho / 10), rho uniform in [-1/2, 1/2) (splitmix64, fixed seed)
        std::vector<float> bw(2 * n);
        uint64_t z = 0x9E3779B97F4A7C15ull ^ (uint64_t)n;
        for (long long i = 0; i < 2 * n; ++i) {
            z += 0x9E3779B97F4A7C15ull;
            uint64_t x = z;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            x ^= x >> 31;
            const double rho = (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
            bw[i] = (float)exp(rho / 10.0);
        }
        cudaError_t e = cudaMemcpyAsync(w->BW, bw.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, c->cap_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->cap_stream);
        if (e != cudaSuccess) return check_cuda(c, e, "butterfly weights");
    }
    w->gp_stride = 2 * n * 2 * n * w->nsplit_elim;
    w->seg_rows = (c->schur_seg > 0 && c->schur_seg < h) ? c->schur_seg : 0;
    w->nseg = w->seg_rows > 0 ? (int)((h + w->seg_rows - 1) / w->seg_rows) : 1;
    WA(w->GP, (w->seg_rows > 0 ? w->seg_rows : h) * w->gp_stride);
    if (w->seg_rows > 0) { WA(w->CK, (long long)(w->nseg - 1) * 2 * n * n); }
    WA(w->O32, 2 * std::max<long long>(ncol, nout) * n);
    WA(w->r, h * ncol * n); WA(w->delta, h * ncol * n);
    WA(w->cb, ncol * n); WA(w->ct, ncol * n);
    WA(w->rnorm, 2 * ncol);
    w->km = c->krylov_m;
    if (w->km > 0) {
        WA(w->KV, (long long)(w->km + 1) * h * ncol * n);
        WA(w->KZ, (long long)w->km * h * ncol * n);
        WA(w->kdot, (long long)(w->km + 1) * w->km * ncol);
        WA(w->ky, (long long)w->km * ncol);
        WA(w->knrm, (long long)w->km * ncol);
    }
#undef WA
    return APF_OK;
}

// G_j = X_j^-1 in place (the block in w->Xre / w->Xim of every design),
// through the symmetric random butterfly transform when it is on and the
// recursion has levels.
int invert_block_b(const Bat &bt, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    MixedWork *w = c->mw;
    const int n = c->nx, nb = bt.n;
    PV X[TC_MAX_BATCH];
    float *tre[TC_MAX_BATCH], *tim[TC_MAX_BATCH], *vre[TC_MAX_BATCH], *vim[TC_MAX_BATCH];
    for (int b = 0; b < nb; ++b) {
        MixedWork *wb = bt.c[b]->mw;
        X[b] = PV{wb->Xre, wb->Xim, n};
        tre[b] = wb->Tre; tim[b] = wb->Tim; vre[b] = wb->Vre; vim[b] = wb->Vim;
    }
    const bool bf = w->bfly && n > leaf_size(w) && n >= 16;
    const dim3 bgrid((n / 4 + 127) / 128, n / 4, nb);
    auto xre = tab<float *>(bt, [&](int b) { return X[b].re; });
    auto xim = tab<float *>(bt, [&](int b) { return X[b].im; });
    if (bf) APF_LAUNCH(c, k_butterfly<false>, bgrid, 128, 0, s, xre, xim, (long long)n, n, (const float *)w->BW);
    int rc = inv32_b(bt, X, n, tre, tim, vre, vim, s);
    if (rc) return rc;
    if (bf) APF_LAUNCH(c, k_butterfly<true>, bgrid, 128, 0, s, xre, xim, (long long)n, n, (const float *)w->BW);
    return APF_OK;
}

// X_row = K_row - G (G: the float32 planes gre/gim of each design, or none) into w->Xre / w->Xim.
static void assemble_b(const Bat &bt, int row, const float *const *gre, const float *const *gim, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    const int n = c->nx;
    dim3 agrid((n / 4 + 255) / 256, n, bt.n);
    APF_LAUNCH(c, k_assemble32, agrid, 256, 0, s, make_grid(c), row,
               tab<const double *>(bt, [&](int b) { return (const double *)bt.c[b]->d_eps; }),
               (const double2 *)c->d_circ, tab<const float *>(bt, [&](int b) { return gre ? gre[b] : nullptr; }),
               tab<const float *>(bt, [&](int b) { return gim ? gim[b] : nullptr; }),
               tab<float *>(bt, [&](int b) { return bt.c[b]->mw->Xre; }),
               tab<float *>(bt, [&](int b) { return bt.c[b]->mw->Xim; }));
}

// Pack every design's G_j (its working block) into its GP slot of row j.
static void pack_gp_b(const Bat &bt, int j, cudaStream_t s) {
    const int n = bt.lead()->nx;
    PackView v[TC_MAX_BATCH];
    PV X[TC_MAX_BATCH];
    __nv_bfloat16 *dst[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) {
        MixedWork *wb = bt.c[b]->mw;
        X[b] = PV{wb->Xre, wb->Xim, n};
        dst[b] = (__nv_bfloat16 *)gp_view(bt.c[b], j).base;
    }
    pack32_b(bt, v, dst, X, n, n, false, true, bt.lead()->mw->nsplit_elim, s);
}

int mixed_eliminate_b(const Bat &bt, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    for (int b = 0; b < bt.n; ++b)
        if (!bt.c[b]->mw) return set_err(bt.c[b], APF_ESTATE, "mixed workspace missing");
    MixedWork *w = c->mw;
    const int n = c->nx;
    const long long nn = (long long)n * n;
    const int K = w->seg_rows;
    const float *xre[TC_MAX_BATCH], *xim[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) { xre[b] = bt.c[b]->mw->Xre; xim[b] = bt.c[b]->mw->Xim; }
    assemble_b(bt, 0, nullptr, nullptr, s);
    for (int j = 0; j < c->h; ++j) {
        int rc = invert_block_b(bt, s);
        if (rc) return rc;
        pack_gp_b(bt, j, s);
        if (K > 0 && j + 1 < c->h && (j + 1) % K == 0) {
            // checkpoint G_j (float32) for the segment that starts at row j + 1
            for (int b = 0; b < bt.n; ++b) {
                MixedWork *wb = bt.c[b]->mw;
                float *ck = wb->CK + (long long)((j + 1) / K - 1) * 2 * nn;
                cudaMemcpyAsync(ck, wb->Xre, sizeof(float) * nn, cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(ck + nn, wb->Xim, sizeof(float) * nn, cudaMemcpyDeviceToDevice, s);
            }
        }
        if (j + 1 < c->h) assemble_b(bt, j + 1, xre, xim, s);
    }
    for (int b = 0; b < bt.n; ++b) bt.c[b]->mw->seg_loaded = K > 0 ? (c->h - 1) / K : -1;
    return APF_OK;
}

int mixed_eliminate(apf_ctx *c, cudaStream_t s) { return mixed_eliminate_b(one(c), s); }

// Recompute the packed inverses of segment `seg` (rows c .. c + seg_rows - 1)
// into the GP slots of every design: X_c = K_c - G_{c-1} from the float32
// checkpoint, then the same inversions and assemblies as the elimination
// (bit-identical results).
int recompute_segment_b(const Bat &bt, int seg, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    MixedWork *w = c->mw;
    const int n = c->nx, K = w->seg_rows;
    const long long nn = (long long)n * n;
    const int r0 = seg * K, r1 = std::min(c->h, r0 + K);
    const float *gre[TC_MAX_BATCH], *gim[TC_MAX_BATCH], *xre[TC_MAX_BATCH], *xim[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) {
        MixedWork *wb = bt.c[b]->mw;
        gre[b] = seg > 0 ? wb->CK + (long long)(seg - 1) * 2 * nn : nullptr;
        gim[b] = seg > 0 ? gre[b] + nn : nullptr;
        xre[b] = wb->Xre;
        xim[b] = wb->Xim;
    }
    assemble_b(bt, r0, seg > 0 ? gre : nullptr, seg > 0 ? gim : nullptr, s);
    for (int j = r0; j < r1; ++j) {
        int rc = invert_block_b(bt, s);
        if (rc) return rc;
        pack_gp_b(bt, j, s);
        if (j + 1 < r1) assemble_b(bt, j + 1, xre, xim, s);
    }
    for (int b = 0; b < bt.n; ++b) bt.c[b]->mw->seg_loaded = seg;
    return APF_OK;
}

// Right-hand side R (written into d_E by the caller), its column norms, and
// the first low-precision solve E = Khat^-1 R.
int mixed_fields_begin_b(const Bat &bt, cudaStream_t s) {
    const double2 *R[TC_MAX_BATCH];
    double2 *E[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) {
        apf_ctx *c = bt.c[b];
        const int ncol = c->cf + c->ca;
        // R = the right-hand side (kept for the residuals) and its column norms, in one pass
        APF_LAUNCH(c, k_colnorm, ncol, 256, 0, s, (const double2 *)c->d_Ew, c->h, ncol, c->nx, c->mw->rnorm, c->d_R);
        R[b] = c->d_R;
        E[b] = c->d_Ew;
    }
    return approx_solve_b(bt, R, E, bt.lead()->cf, s);
}

int mixed_fields_begin(apf_ctx *c, cudaStream_t s) { return mixed_fields_begin_b(one(c), s); }

static int resid_body(apf_ctx *c, cudaStream_t s) {
    MixedWork *w = c->mw;
    int ncol = c->cf + c->ca;
    residual(c, c->d_Ew, w->r, s);
    APF_LAUNCH(c, k_colnorm, ncol, 256, 0, s, w->r, c->h, ncol, c->nx, w->rnorm + ncol, (double2 *)nullptr);
    return APF_OK;
}

// E += Khat^-1 r for every design of the batch.
static int correct_b(const Bat &bt, cudaStream_t s) {
    const double2 *r[TC_MAX_BATCH];
    double2 *d[TC_MAX_BATCH];
    for (int b = 0; b < bt.n; ++b) {
        r[b] = bt.c[b]->mw->r;
        d[b] = bt.c[b]->mw->delta;
    }
    apf_ctx *c0 = bt.lead();
    int rc = approx_solve_b(bt, r, d, c0->cf + c0->ca, s);
    if (rc) return rc;
    for (int b = 0; b < bt.n; ++b) {
        apf_ctx *c = bt.c[b];
        const long long total = (long long)(c->cf + c->ca) * c->nx * c->h;
        APF_LAUNCH(c, k_axpy, (unsigned)((total + 255) / 256), 256, 0, s, c->d_Ew, c->mw->delta, total);
    }
    return APF_OK;
}

static int correct_body(apf_ctx *c, cudaStream_t s) { return correct_b(one(c), s); }

// Diagnostics: APF_IR_VERBOSE=1 prints the residual of every refinement step.
static const bool g_ir_verbose = [] {
    const char *e = getenv("APF_IR_VERBOSE");
    return e && e[0] == '1';
}();

// K E (the slab operator in float64) into out.
static int apply_K(apf_ctx *c, const double2 *E, double2 *out, cudaStream_t s) {
    MixedWork *w = c->mw;
    const int ncol = c->cf + c->ca, nx = c->nx;
    const long long L = (long long)ncol * nx;
    int logn = 0;
    while ((1 << logn) < nx) ++logn;
    const int threads = nx / 2 < 256 ? nx / 2 : 256;
    const int smem = nx * (int)sizeof(double2);
    APF_LAUNCH(c, k_circ_apply, ncol, threads, smem, s, E, w->cb, nx, logn, c->d_modes, c->d_tw);
    APF_LAUNCH(c, k_circ_apply, ncol, threads, smem, s, E + (c->h - 1) * L, w->ct, nx, logn, c->d_modes + nx,
               c->d_tw);
    GridDev g = make_grid(c);
    dim3 grid((nx + 255) / 256, ncol, c->h);
    APF_LAUNCH(c, k_residual, grid, 256, 0, s, g, c->d_eps, E, (const double2 *)nullptr, w->cb, w->ct, out, ncol);
    return APF_OK;
}

// min || beta e1 - H y || for one column by complex Givens rotations; H is
// (m+1) x m upper Hessenberg, H[i][j] at h[i * m + j].
static void hessenberg_lsq(int m, std::vector<std::complex<double>> &h, double beta, std::complex<double> *y) {
    std::vector<std::complex<double>> g(m + 1, 0.0), cs(m), sn(m);
    std::vector<double> cr(m);
    g[0] = beta;
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i < j; ++i) {
            const std::complex<double> a = h[i * m + j], b = h[(i + 1) * m + j];
            h[i * m + j] = cr[i] * a + sn[i] * b;
            h[(i + 1) * m + j] = -std::conj(sn[i]) * a + cr[i] * b;
        }
        const std::complex<double> a = h[j * m + j], b = h[(j + 1) * m + j];
        const double na = std::abs(a), nb = std::abs(b);
        if (nb == 0.0) {
            cr[j] = 1.0; sn[j] = 0.0;
        } else if (na == 0.0) {
            cr[j] = 0.0; sn[j] = std::conj(b) / nb;
        } else {
            const double nr = std::sqrt(na * na + nb * nb);
            cr[j] = na / nr;
            sn[j] = (a / na) * std::conj(b) / nr;
        }
        h[j * m + j] = cr[j] * a + sn[j] * b;
        h[(j + 1) * m + j] = 0.0;
        const std::complex<double> g0 = g[j], g1 = g[j + 1];
        g[j] = cr[j] * g0 + sn[j] * g1;
        g[j + 1] = -std::conj(sn[j]) * g0 + cr[j] * g1;
    }
    for (int j = m - 1; j >= 0; --j) {
        std::complex<double> t = g[j];
        for (int k = j + 1; k < m; ++k) t -= h[j * m + k] * y[k];
        y[j] = std::abs(h[j * m + j]) > 0.0 ? t / h[j * m + j] : 0.0;
    }
}

// Float64 refinement by restarted GMRES(m), right-preconditioned by the
// low-precision factorization Khat^-1 (a fixed linear operator), one Krylov
// space per right-hand-side column: from the true residual r = R - K E,
// V_0 = r / ||r||; Z_j = Khat^-1 V_j, W = K Z_j orthogonalised against
// V_0..V_j (modified Gram-Schmidt, per-column coefficients kept on the
// device), V_{j+1} = W / ||W||; then E += sum_j y_j Z_j with y the
// per-column least-squares solution of the (m+1) x m Hessenberg system.
// The stopping rule and the iteration count (preconditioner applications)
// are those of the plain refinement.
static int mixed_refine_gmres(apf_ctx *c, cudaStream_t s) {
    MixedWork *w = c->mw;
    const int m = w->km, ncol = c->cf + c->ca, nx = c->nx;
    const long long L = (long long)c->h * ncol * nx;
    const dim3 fgrid((nx + 255) / 256, ncol, c->h);
    std::vector<double> nr(ncol), ne(ncol), hn((size_t)m * ncol);
    std::vector<double2> hd((size_t)(m + 1) * m * ncol), yh((size_t)m * ncol);
    std::vector<std::complex<double>> H((size_t)(m + 1) * m), y(m);
    int iters = 0, rc, rising = 0;
    double ratio = 0.0, prev = INFINITY;
    cudaMemcpyAsync(nr.data(), w->rnorm, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s);
    for (;;) {
        residual(c, c->d_Ew, w->r, s);
        APF_LAUNCH(c, k_colnorm, ncol, 256, 0, s, w->r, c->h, ncol, nx, w->rnorm + ncol, (double2 *)nullptr);
        cudaMemcpyAsync(ne.data(), w->rnorm + ncol, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return check_cuda(c, e, "refinement");
        if (c->prof_on && iters == 0) prof_collect_range(c, c->g_main[c->lay].prof_lo, c->g_main[c->lay].prof_hi);
        ratio = 0.0;
        for (int i = 0; i < ncol; ++i) ratio = std::max(ratio, sqrt(ne[i] / std::max(nr[i], 1e-300)));
        if (g_ir_verbose)
            fprintf(stderr, "apf refinement (GMRES(%d)): %d preconditioner applications, max relative residual %.3e\n",
                    m, iters, ratio);
        if (!(ratio == ratio)) { ratio = INFINITY; break; }
        if (ratio <= c->ir_tol || iters >= c->ir_max) break;
        rising = ratio > prev ? rising + 1 : 0;
        if (rising >= 2) break;
        prev = ratio;
        // Arnoldi on K Khat^-1 from V_0 = r / ||r||
        APF_LAUNCH(c, k_colscale, fgrid, 256, 0, s, w->KV, w->r, w->rnorm + ncol, ncol, nx);
        for (int j = 0; j < m; ++j) {
            double2 *Vj = w->KV + j * L, *Wn = w->KV + (j + 1) * L, *Zj = w->KZ + j * L;
            if ((rc = approx_solve(c, Vj, Zj, ncol, s))) return rc;
            apply_K(c, Zj, Wn, s);
            for (int i = 0; i <= j; ++i) {
                double2 *hij = w->kdot + ((long long)j * (m + 1) + i) * ncol;
                APF_LAUNCH(c, k_coldot, ncol, 256, 0, s, w->KV + i * L, Wn, c->h, ncol, nx, hij);
                APF_LAUNCH(c, k_colaxpy, fgrid, 256, 0, s, Wn, w->KV + i * L, hij, -1.0, ncol, nx);
            }
            APF_LAUNCH(c, k_colnorm, ncol, 256, 0, s, Wn, c->h, ncol, nx, w->knrm + (long long)j * ncol,
                       (double2 *)nullptr);
            APF_LAUNCH(c, k_colscale, fgrid, 256, 0, s, Wn, Wn, w->knrm + (long long)j * ncol, ncol, nx);
        }
        cudaMemcpyAsync(hd.data(), w->kdot, sizeof(double2) * hd.size(), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hn.data(), w->knrm, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return check_cuda(c, e, "arnoldi");
        for (int col = 0; col < ncol; ++col) {
            std::fill(H.begin(), H.end(), std::complex<double>(0.0, 0.0));
            for (int j = 0; j < m; ++j) {
                for (int i = 0; i <= j; ++i) {
                    const double2 v = hd[((size_t)j * (m + 1) + i) * ncol + col];
                    H[(size_t)i * m + j] = std::complex<double>(v.x, v.y);
                }
                H[(size_t)(j + 1) * m + j] = std::sqrt(std::max(hn[(size_t)j * ncol + col], 0.0));
            }
            hessenberg_lsq(m, H, std::sqrt(std::max(ne[col], 0.0)), y.data());
            for (int j = 0; j < m; ++j) yh[(size_t)j * ncol + col] = make_double2(y[j].real(), y[j].imag());
        }
        cudaMemcpyAsync(w->ky, yh.data(), sizeof(double2) * yh.size(), cudaMemcpyHostToDevice, s);
        for (int j = 0; j < m; ++j)
            APF_LAUNCH(c, k_colaxpy, fgrid, 256, 0, s, c->d_Ew, w->KZ + j * L, w->ky + (long long)j * ncol, 1.0,
                       ncol, nx);
        iters += m;
    }
    c->stats.refine_iters = iters;
    c->stats.residual = ratio;
    return ratio <= c->ir_tol ? APF_OK : APF_ENOCONV;
}

// Float64 iterative refinement: r = R - K E, E += Khat^-1 r until
// max_c ||r_c|| / ||R_c|| <= tol (or max_iters corrections).
int mixed_refine(apf_ctx *c, cudaStream_t s) {
    MixedWork *w = c->mw;
    if (w->km > 0) return mixed_refine_gmres(c, s);
    int ncol = c->cf + c->ca;
    std::vector<double> nr(ncol), ne(ncol);
    int iters = 0, rc, rising = 0;
    double ratio = 0.0, prev = INFINITY;
    for (;;) {
        if ((rc = run_graph(c, c->g_resid[c->lay], s, resid_body))) return rc;
        cudaMemcpyAsync(nr.data(), w->rnorm, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(ne.data(), w->rnorm + ncol, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return check_cuda(c, e, "refinement");
        if (c->prof_on) {
            const GraphSlot &g = iters == 0 ? c->g_main[c->lay] : c->g_correct[c->lay];
            prof_collect_range(c, g.prof_lo, g.prof_hi);
        }
        ratio = 0.0;
        for (int i = 0; i < ncol; ++i) ratio = std::max(ratio, sqrt(ne[i] / std::max(nr[i], 1e-300)));
        if (g_ir_verbose) fprintf(stderr, "apf refinement: iteration %d, max relative residual %.3e\n", iters, ratio);
        if (!(ratio == ratio)) { ratio = INFINITY; break; }
        if (ratio <= c->ir_tol || iters >= c->ir_max) break;
        // diverging: the residual grew on two consecutive sweeps
        rising = ratio > prev ? rising + 1 : 0;
        if (rising >= 2) break;
        prev = ratio;
        if ((rc = run_graph(c, c->g_correct[c->lay], s, correct_body))) return rc;
        ++iters;
    }
    c->stats.refine_iters = iters;
    c->stats.residual = ratio;
    return ratio <= c->ir_tol ? APF_OK : APF_ENOCONV;
}

// Gradient contraction with tensor-core products: Q_j = Gamma F_j, then
// g_j(x) = 2 k^2 Re sum_b Phi_j[b][x] Q_j[b][x] in float64.
// Gradient contraction with tensor-core products for every design of the
// batch: Q_j = Gamma F_j, then g_j(x) = 2 k^2 Re sum_b Phi_j[b][x] Q_j[b][x] in
// float64.  Gamma[b]: the design's n_out x n_in Gamma on the device.
int mixed_gradient_b(const Bat &bt, const double2 *const *Gamma, cudaStream_t s) {
    apf_ctx *c = bt.lead();
    MixedWork *w = c->mw;
    const int nin = c->nin, nout = c->nout, ncol = nin + nout;
    const int nx = c->nx, ns = w->nsplit_grad, nb = bt.n;
    const long long L = (long long)ncol * nx;
    PackView pa[TC_MAX_BATCH], pb[TC_MAX_BATCH];
    __nv_bfloat16 *padst[TC_MAX_BATCH], *pbdst[TC_MAX_BATCH];
    PV Q[TC_MAX_BATCH];
    const double2 *src[TC_MAX_BATCH];
    for (int b = 0; b < nb; ++b) {
        MixedWork *wb = bt.c[b]->mw;
        padst[b] = wb->PA;
        pbdst[b] = wb->PB;
        Q[b] = PV{wb->O32, wb->O32 + (long long)nout * nx, nx};
    }
    pack64A_b(bt, pa, padst, Gamma, nullptr, nin, nout, nin, ns, s);
    for (int j = 0; j < c->h; ++j) {
        for (int b = 0; b < nb; ++b) src[b] = bt.c[b]->d_E + j * L;
        pack64BT_b(bt, pb, pbdst, src, nx, nx, nin, ns, s);
        int rc = gemm_b(bt, pa, pb, ns, nout, 2 * nx, nx, 1.f, 0.f, Q, nullptr, s);
        if (rc) return rc;
        APF_LAUNCH(c, k_grad_rowdot32, dim3((nx + 31) / 32, 1, nb), 256, 0, s,
                   tab<const double2 *>(bt, [&](int b) { return (const double2 *)bt.c[b]->d_E; }),
                   tab<const float *>(bt, [&](int b) { return (const float *)Q[b].re; }),
                   tab<const float *>(bt, [&](int b) { return (const float *)Q[b].im; }), j, nx, nin, nout,
                   c->k * c->k, tab<double *>(bt, [&](int b) { return bt.c[b]->d_grad; }));
    }
    return APF_OK;
}

int mixed_gradient(apf_ctx *c, const double2 *Gamma, cudaStream_t s) { return mixed_gradient_b(one(c), &Gamma, s); }

// Refinement of a batch of designs (no captured graphs): every sweep checks
// the residual of each design, and designs still above tolerance take one
// more correction, all of them in the same launches.  The stopping rule per
// design is that of mixed_refine.  rc[b]: APF_OK or APF_ENOCONV.
int mixed_refine_b(const Bat &bt, cudaStream_t s, int *rcs) {
    const int nb = bt.n;
    apf_ctx *c0 = bt.lead();
    const int ncol = c0->cf + c0->ca;
    std::vector<std::vector<double>> nr(nb, std::vector<double>(ncol)), ne(nb, std::vector<double>(ncol));
    std::vector<int> iters(nb, 0), rising(nb, 0), active(nb, 1);
    std::vector<double> ratio(nb, 0.0), prev(nb, INFINITY);
    for (;;) {
        for (int b = 0; b < nb; ++b) {
            if (!active[b]) continue;
            apf_ctx *c = bt.c[b];
            resid_body(c, s);
            cudaMemcpyAsync(nr[b].data(), c->mw->rnorm, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(ne[b].data(), c->mw->rnorm + ncol, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s);
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return check_cuda(c0, e, "refinement");
        Bat next;
        next.n = 0;
        for (int b = 0; b < nb; ++b) {
            if (!active[b]) continue;
            apf_ctx *c = bt.c[b];
            double r = 0.0;
            for (int i = 0; i < ncol; ++i) r = std::max(r, sqrt(ne[b][i] / std::max(nr[b][i], 1e-300)));
            ratio[b] = (r == r) ? r : INFINITY;
            bool stop = !(r == r) || r <= c->ir_tol || iters[b] >= c->ir_max;
            if (!stop) {
                rising[b] = r > prev[b] ? rising[b] + 1 : 0;
                stop = rising[b] >= 2;
            }
            prev[b] = r;
            if (stop) active[b] = 0;
            else next.c[next.n++] = c;
        }
        if (next.n == 0) break;
        int rc = correct_b(next, s);
        if (rc) return rc;
        for (int b = 0; b < nb; ++b)
            if (active[b]) ++iters[b];
    }
    for (int b = 0; b < nb; ++b) {
        apf_ctx *c = bt.c[b];
        c->stats.refine_iters = iters[b];
        c->stats.residual = ratio[b];
        rcs[b] = ratio[b] <= c->ir_tol ? APF_OK : APF_ENOCONV;
    }
    return APF_OK;
}

// Entry points for a batch of contexts (apf_solve_S_grad_batch).
static Bat make_bat(apf_ctx *const *cs, int nb) {
    Bat bt;
    bt.n = nb;
    for (int b = 0; b < nb; ++b) bt.c[b] = cs[b];
    return bt;
}
int mixed_eliminate_n(apf_ctx *const *cs, int nb, cudaStream_t s) { return mixed_eliminate_b(make_bat(cs, nb), s); }
int mixed_fields_begin_n(apf_ctx *const *cs, int nb, cudaStream_t s) {
    return mixed_fields_begin_b(make_bat(cs, nb), s);
}
int mixed_refine_n(apf_ctx *const *cs, int nb, cudaStream_t s, int *rcs) {
    return mixed_refine_b(make_bat(cs, nb), s, rcs);
}
int mixed_gradient_n(apf_ctx *const *cs, int nb, cudaStream_t s) {
    const double2 *g[TC_MAX_BATCH];
    for (int b = 0; b < nb; ++b) g[b] = cs[b]->d_Gam;
    return mixed_gradient_b(make_bat(cs, nb), g, s);
}
// Settings that must agree across the designs of a batch (the launches are shared).
bool mixed_batch_compatible(const apf_ctx *a, const apf_ctx *b) {
    const MixedWork *x = a->mw, *y = b->mw;
    if (!x || !y) return false;
    return x->nsplit_elim == y->nsplit_elim && x->nsplit_grad == y->nsplit_grad && x->leaf == y->leaf &&
           x->leaf_variant == y->leaf_variant && x->seg_rows == y->seg_rows && x->bfly == y->bfly && x->km == 0 &&
           y->km == 0;
}

// ---------------------------------------------------------------------------
// Test hooks (not part of the public ABI in include/): exercise the packing +
// tensor-core GEMM and the mixed recursive inversion in isolation.  They
// allocate their own temporaries.
// ---------------------------------------------------------------------------
extern "C" int apf_debug_cgemm(apf_ctx *c, int m, int n, int k, const float *Are, const float *Aim,
                               const float *Bre, const float *Bim, float *Cre, float *Cim, int nsplit) {
    if (!c) return APF_EINVAL;
    SolveGate gate(c->device);
    if (m < 1 || n < 1 || k < 1 || nsplit < 1 || nsplit > 3) return APF_EINVAL;
    cudaSetDevice(c->device);
    long long kp = round_up(2LL * k, 64);
    __nv_bfloat16 *pa = nullptr, *pb = nullptr;
    if (cudaMalloc(&pa, sizeof(__nv_bfloat16) * m * kp * nsplit) != cudaSuccess) return APF_ENOMEM;
    if (cudaMalloc(&pb, sizeof(__nv_bfloat16) * 2LL * n * kp * nsplit) != cudaSuccess) { cudaFree(pa); return APF_ENOMEM; }
    int *flags = c->d_flags;
    int *tmpflags = nullptr;
    if (!flags) { cudaMalloc(&tmpflags, 16); cudaMemset(tmpflags, 0, 16); c->d_flags = tmpflags; }
    cudaStream_t s = 0;
    PackView A = pack32(c, pa, PV{(float *)Are, (float *)Aim, k}, m, k, false, false, nsplit, s);
    PackView B = pack32(c, pb, PV{(float *)Bre, (float *)Bim, n}, n, k, true, true, nsplit, s);
    int rc = tc_gemm(c, A, B, nsplit, m, 2 * n, n, 1.f, 0.f, Cre, Cim, n, nullptr, nullptr, 0, s);
    cudaError_t e = cudaDeviceSynchronize();
    if (c->prof_on) prof_collect(c);  // GEMM event timings of this call
    int fl = 0;
    cudaMemcpy(&fl, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (tmpflags) { cudaFree(tmpflags); c->d_flags = nullptr; }
    cudaFree(pa);
    cudaFree(pb);
    if (rc) return rc;
    if (e != cudaSuccess) return check_cuda(c, e, "debug cgemm");
    if (fl & FLAG_TIMEOUT) return set_err(c, APF_ETIMEOUT, "tc_gemm wait gave up");
    return APF_OK;
}

// In-place inverse of an n x n complex-symmetric planar float32 matrix using
// the workspace of a prepared mixed-precision context (n <= its nx).
extern "C" int apf_debug_inv32(apf_ctx *c, int n, float *re, float *im, int leaf) {
    if (!c) return APF_EINVAL;
    SolveGate gate(c->device);
    if (!c || !c->mw || n < 1 || n > c->nx || (n & (n - 1))) return APF_EINVAL;
    cudaSetDevice(c->device);
    int old = c->mw->leaf, oldv = c->mw->leaf_variant;
    // leaf = block size + 1000 * kernel variant (test and tuning hook);
    // + 100000: through the symmetric random butterfly transform
    const bool bf = leaf >= 100000 && n >= 16;
    leaf %= 100000;
    if (leaf > 0) { c->mw->leaf = leaf % 1000; c->mw->leaf_variant = leaf / 1000; }
    cudaMemset(c->d_flags, 0, 16);
    const dim3 bgrid((n / 4 + 127) / 128, n / 4);
    Tab<float *> tre{}, tim{};
    tre.v[0] = re;
    tim.v[0] = im;
    if (bf) APF_LAUNCH(c, k_butterfly<false>, bgrid, 128, 0, (cudaStream_t)0, tre, tim, (long long)n, n, (const float *)c->mw->BW);
    int rc = inv32(c, PV{re, im, n}, n, c->mw->Tre, c->mw->Tim, c->mw->Vre, c->mw->Vim, 0);
    if (bf && rc == APF_OK)
        APF_LAUNCH(c, k_butterfly<true>, bgrid, 128, 0, (cudaStream_t)0, tre, tim, (long long)n, n, (const float *)c->mw->BW);
    cudaError_t e = cudaDeviceSynchronize();
    c->mw->leaf = old;
    c->mw->leaf_variant = oldv;
    if (rc) return rc;
    if (e != cudaSuccess) return check_cuda(c, e, "debug inv32");
    int fl = 0;
    cudaMemcpy(&fl, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (fl & FLAG_TIMEOUT) return set_err(c, APF_ETIMEOUT, "tc_gemm wait gave up");
    if (fl & FLAG_SINGULAR) return set_err(c, APF_ESINGULAR, "singular leaf");
    return APF_OK;
}
