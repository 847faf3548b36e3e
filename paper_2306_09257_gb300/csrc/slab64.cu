// Float64 slab elimination: assembly of the slab Schur blocks X_j, a complex
// float64 GEMM, diagonal-block inversion, and the recursive inversion of the
// complex-symmetric X_j.
//
// In the pixel basis the slab rows j = 0..h-1 form a block-tridiagonal system
// with diagonal blocks K_j = T_x + 2 I - k^2 diag(eps_j) + 2 I (T_x the
// periodic second difference; the two y-couplings give the other 2 I),
// plus the boundary Schur blocks Sigma_bot on row 0 and Sigma_top on row h-1
// (circulants, diagonal in the Fourier basis), and off-diagonal blocks -I.
// Forward block elimination: X_0 = K_0, X_j = K_j - X_{j-1}^-1 (the Schur
// complement of the rows below; paper Sec. 2: S is a Schur complement of
// the augmented K, obtained here block row by block row).  Every X_j is
// complex symmetric (reciprocity, A = A^T), which the inversion exploits.
#include "apf_internal.h"
#include "leaf.cuh"

namespace {

__global__ void k_assemble64(GridDev g, int row, const double *eps, const double2 *circ,
                             const double2 *Gprev, double2 *X) {
    int xp = blockIdx.x * blockDim.x + threadIdx.x;
    int x = blockIdx.y;
    int n = g.nx;
    if (xp >= n) return;
    double2 v = cmk(0.0, 0.0);
    if (xp == x) v.x += 4.0 - g.k * g.k * eps[(long long)row * n + x];
    if (xp == (x + 1) % n) v.x -= 1.0;
    if (xp == (x + n - 1) % n) v.x -= 1.0;
    int d = (x - xp + n) % n;
    if (row == 0) v = cadd(v, circ[d]);
    if (row == g.h - 1) v = cadd(v, circ[n + d]);
    long long idx = (long long)x * n + xp;
    if (Gprev) v = csub(v, Gprev[idx]);
    X[idx] = v;
}

// C = alpha op(A) op(B) + beta C, row-major complex float64, batched over
// blockIdx.z.  64x64 tile per block, 8-deep k slices, 4x4 outputs per thread.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_zgemm(int M, int N, int K, double2 alpha,
                                              const double2 *__restrict__ A, long long lda, long long sA,
                                              const double2 *__restrict__ B, long long ldb, long long sB,
                                              double2 beta, double2 *C, long long ldc, long long sC) {
    constexpr int BM = 64, BN = 64, BK = 8;
    __shared__ double2 As[BK][BM];
    __shared__ double2 Bs[BK][BN];
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmk(0.0, 0.0);
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int e = threadIdx.x + r * 256;  // 0..511
            int kk, ii;
            if (TA) { ii = e & 63; kk = e >> 6; }   // contiguous along m
            else { kk = e & 7; ii = e >> 3; }       // contiguous along k
            int gi = m0 + ii, gk = k0 + kk;
            double2 v = cmk(0.0, 0.0);
            if (gi < M && gk < K) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
            As[kk][ii] = v;
            int jj;
            if (TB) { kk = e & 7; jj = e >> 3; }    // contiguous along k
            else { jj = e & 63; kk = e >> 6; }      // contiguous along n
            int gj = n0 + jj;
            gk = k0 + kk;
            v = cmk(0.0, 0.0);
            if (gj < N && gk < K) v = TB ? B[(long long)gj * ldb + gk] : B[(long long)gk * ldb + gj];
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
                    acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
    bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gi = m0 + ty + 16 * i;
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gj = n0 + tx + 16 * j;
            if (gj >= N) continue;
            double2 v = cmul(alpha, acc[i][j]);
            long long idx = (long long)gi * ldc + gj;
            if (use_beta) v = cadd(v, cmul(beta, C[idx]));
            C[idx] = v;
        }
    }
}

// In-place inverse of an n x n (n <= 64) block by Gauss-Jordan elimination
// with partial (row) pivoting, in shared memory.  Row interchanges during the
// sweep become column interchanges of the result, undone in reverse order.
__global__ void __launch_bounds__(256) k_leaf_inv64(double2 *X, int n, long long ld, int *flags) {
    extern __shared__ double2 a[];  // n*n
    __shared__ double2 colk[64];
    __shared__ int piv[64];
    __shared__ int s_p;
    __shared__ double2 s_inv;
    int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) a[e] = X[(long long)(e / n) * ld + (e % n)];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                double v = cabs2(a[i * n + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                double ob = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                s_p = bi;
                piv[k] = bi;
                if (!(best > 0.0) || !isfinite(best)) atomicOr(flags, FLAG_SINGULAR);
            }
        }
        __syncthreads();
        int p = s_p;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                double2 t = a[k * n + j];
                a[k * n + j] = a[p * n + j];
                a[p * n + j] = t;
            }
            __syncthreads();
        }
        if (tid == 0) s_inv = cinv(a[k * n + k]);
        __syncthreads();
        double2 inv = s_inv;
        for (int j = tid; j < n; j += nt) {
            a[k * n + j] = (j == k) ? inv : cmul(a[k * n + j], inv);
        }
        for (int i = tid; i < n; i += nt) colk[i] = a[i * n + k];
        __syncthreads();
        for (int e = tid; e < n * n; e += nt) {
            int i = e / n, j = e - i * n;
            if (i == k) continue;
            double2 f = colk[i];
            if (j == k) a[e] = cscale(cmul(f, inv), -1.0);
            else a[e] = csub(a[e], cmul(f, a[k * n + j]));
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k) {
            for (int i = tid; i < n; i += nt) {
                double2 t = a[i * n + k];
                a[i * n + k] = a[i * n + p];
                a[i * n + p] = t;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt) X[(long long)(e / n) * ld + (e % n)] = a[e];
}

template <int NB>
__global__ void __launch_bounds__(NB * 4) k_leaf64(double2 *X, long long ld, int *flags) {
    LeafIO<double, false> io{nullptr, nullptr, X, ld};
    leaf_gj<double, NB, false>(io, flags);
}

// C block <- -V, B block <- -V^T  (the off-diagonal blocks of the inverse).
__global__ void k_neg_offdiag(double2 *Bblk, double2 *Cblk, long long ld, const double2 *V, int h) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= h) return;
    double2 v = V[(long long)i * h + j];
    Cblk[(long long)i * ld + j] = cscale(v, -1.0);
    Bblk[(long long)j * ld + i] = cscale(v, -1.0);
}

__global__ void k_add2(double2 *T, const double2 *a, const double2 *b, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) T[i] = cadd(a[i], b[i]);
}

__global__ void k_copy(double2 *d, const double2 *s, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) d[i] = s[i];
}

constexpr int LEAF64 = 32;

}  // namespace

void launch_assemble64(apf_ctx *c, int row, double2 *X, const double2 *Gprev, cudaStream_t s) {
    GridDev g = make_grid(c);
    dim3 grid((c->nx + 255) / 256, c->nx);
    APF_LAUNCH(c, k_assemble64, grid, 256, 0, s, g, row, c->d_eps, c->d_circ, Gprev, X);
}

void zgemm(apf_ctx *c, bool ta, bool tb, int M, int N, int K, double2 alpha, const double2 *A, long long lda,
           long long sA, const double2 *B, long long ldb, long long sB, double2 beta, double2 *C, long long ldc,
           long long sC, int batch, cudaStream_t s) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
    if (!ta && !tb) APF_LAUNCH(c, (k_zgemm<false, false>), grid, 256, 0, s, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    else if (ta && !tb) APF_LAUNCH(c, (k_zgemm<true, false>), grid, 256, 0, s, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    else if (!ta && tb) APF_LAUNCH(c, (k_zgemm<false, true>), grid, 256, 0, s, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    else APF_LAUNCH(c, (k_zgemm<true, true>), grid, 256, 0, s, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
}

// X <- X^-1 in place for complex-symmetric X (n a power of two), by the
// 2x2 block Schur recursion
//   [A B; C D]^-1 = [Ai + T^T V, -V^T; -V, Si],  T = C Ai, S = D - T B,
//   Si = S^-1, V = Si T,
// which uses B = C^T and Ai = Ai^T, so four GEMMs per level.  Pivoting is
// confined to the diagonal leaf blocks.
void invert_sym64(apf_ctx *c, double2 *X, int n, long long ld, double2 *scr1, double2 *scr2, cudaStream_t s) {
    if (n <= LEAF64) {
        if (n == 32) APF_LAUNCH(c, k_leaf64<32>, 1, 128, leaf_smem_bytes<32>(16), s, X, ld, c->d_flags);
        else if (n == 16) APF_LAUNCH(c, k_leaf64<16>, 1, 64, leaf_smem_bytes<16>(16), s, X, ld, c->d_flags);
        else APF_LAUNCH(c, k_leaf_inv64, 1, 256, n * n * (int)sizeof(double2), s, X, n, ld, c->d_flags);
        return;
    }
    int h = n / 2;
    double2 *A = X, *B = X + h, *C = X + (long long)h * ld, *D = X + (long long)h * ld + h;
    double2 *T = scr1, *V = scr2;
    long long hh = (long long)h * h;
    const double2 one = cmk(1, 0), zero = cmk(0, 0), mone = cmk(-1, 0);
    invert_sym64(c, A, h, ld, scr1 + hh, scr2 + hh, s);
    zgemm(c, false, false, h, h, h, one, C, ld, 0, A, ld, 0, zero, T, h, 0, 1, s);
    zgemm(c, false, false, h, h, h, mone, T, h, 0, B, ld, 0, one, D, ld, 0, 1, s);
    invert_sym64(c, D, h, ld, scr1 + hh, scr2 + hh, s);
    zgemm(c, false, false, h, h, h, one, D, ld, 0, T, h, 0, zero, V, h, 0, 1, s);
    zgemm(c, true, false, h, h, h, one, T, h, 0, V, h, 0, one, A, ld, 0, 1, s);
    dim3 grid((h + 255) / 256, h);
    APF_LAUNCH(c, k_neg_offdiag, grid, 256, 0, s, B, C, ld, V, h);
}

void launch_copy(apf_ctx *c, double2 *dst, const double2 *src, long long n, cudaStream_t s) {
    APF_LAUNCH(c, k_copy, (unsigned)((n + 255) / 256), 256, 0, s, dst, src, n);
}

void launch_add(apf_ctx *c, double2 *T, const double2 *a, const double2 *b, long long n, cudaStream_t s) {
    APF_LAUNCH(c, k_add2, (unsigned)((n + 255) / 256), 256, 0, s, T, a, b, n);
}

void launch_zero(apf_ctx *c, void *dst, long long bytes, cudaStream_t s) {
    (void)c;
    cudaMemsetAsync(dst, 0, (size_t)bytes, s);
}

void slab64_init_attrs() {
    cudaFuncSetAttribute(k_leaf_inv64, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * (int)sizeof(double2));
}
