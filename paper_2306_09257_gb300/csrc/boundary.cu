// Per-Fourier-mode boundary elimination, channel coefficients, right-hand
// sides, and a float64 FFT.
//
// Rows outside the design slab have x-uniform permittivity, so in the Fourier
// basis u_m(x) = exp(2 pi i m x/nx)/sqrt(nx) every such row of A is diagonal:
// for order m the block-tridiagonal A restricted to those rows is a scalar
// tridiagonal recurrence along y.  Eliminating the substrate + bottom PML
// (from the bottom wall up) and the cladding + top PML (from the top wall
// down) leaves, on the first and last slab rows, diagonal (in m) Schur terms
// sigma_bot[m], sigma_top[m]; the input source row's coefficient reaches the
// first slab row multiplied by fac_bot[m]; and the field on the last slab row
// reaches the output row multiplied by tau[m].  This is the structured
// replacement of the sparse partial factorization of K = [A, B; C, D]
// (paper Sec. 2, first paragraph): S = C A^-1 B without assembling A.
#include "apf_internal.h"

#include <math.h>

namespace {

__device__ double2 stretch_at(const GridDev &g, double y) {
    double lo = g.npml_bot - 0.5, hi = g.ny - g.npml_top - 0.5;
    double L, d, eps;
    if (y < lo) {
        L = g.npml_bot; d = lo - y; eps = g.eps_sub;
    } else if (y > hi) {
        L = g.npml_top; d = y - hi; eps = g.eps_clad;
    } else {
        return cmk(1.0, 0.0);
    }
    double alpha = -(g.power + 1.0) * log(g.R0) / (2.0 * g.k * sqrt(eps) * L);
    return cmk(1.0, alpha * pow(d / L, g.power));
}

// Stretch table: st[j] = s_j (integer rows), st[ny + 1 + j] = 1 / s_{j - 1/2}
// for j = 0..ny (half-integer rows, Dirichlet walls beyond the ends).
__global__ void k_stretch_table(GridDev g, double2 *st) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > g.ny) return;
    if (j < g.ny) st[j] = stretch_at(g, (double)j);
    st[g.ny + 1 + j] = cinv(stretch_at(g, j - 0.5));
}

// Diagonal of row j for Fourier order with eigenvalue lam of -d2/dx2:
// s_j (lam - k^2 eps) + 1/s_{j+1/2} + 1/s_{j-1/2}.
__device__ __forceinline__ double2 row_diag(const GridDev &g, const double2 *st, int j, double lam, double eps) {
    double2 t = cscale(st[j], lam - g.k * g.k * eps);
    t = cadd(t, st[g.ny + 1 + j + 1]);
    t = cadd(t, st[g.ny + 1 + j]);
    return t;
}

__global__ void k_boundary_sweep(GridDev g, const double2 *st, double2 *modes) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.nx) return;
    const double2 *ish = st + g.ny + 1;  // ish[j] = 1 / s_{j - 1/2}
    double sp = sinpi((double)m / (double)g.nx);
    double lam = 4.0 * sp * sp;
    // bottom: substrate + PML, rows 0 .. j0-1, eliminated upward
    double2 dt = row_diag(g, st, 0, lam, g.eps_sub);
    double2 fac = cmk(1.0, 0.0);
    for (int j = 1; j < g.j0; ++j) {
        double2 c = ish[j];
        double2 idt = cinv(dt);
        if (j - 1 >= g.jsrc) fac = cmul(fac, cmul(c, idt));
        dt = csub(row_diag(g, st, j, lam, g.eps_sub), cmul(cmul(c, c), idt));
    }
    double2 c0 = ish[g.j0];
    double2 idt0 = cinv(dt);
    fac = cmul(fac, cmul(c0, idt0));
    double2 sig_bot = cscale(cmul(cmul(c0, c0), idt0), -1.0);
    // top: cladding + PML, rows ny-1 .. j0+h, eliminated downward
    double2 dd = row_diag(g, st, g.ny - 1, lam, g.eps_clad);
    double2 tau = cmk(1.0, 0.0);
    for (int j = g.ny - 2; j >= g.j0 + g.h; --j) {
        double2 c = ish[j + 1];
        dd = csub(row_diag(g, st, j, lam, g.eps_clad), cdiv(cmul(c, c), dd));
        if (j <= g.jout) tau = cmul(tau, cdiv(ish[j], dd));
    }
    double2 c1 = ish[g.j0 + g.h];
    double2 sig_top = cscale(cdiv(cmul(c1, c1), dd), -1.0);
    modes[m] = sig_bot;
    modes[g.nx + m] = sig_top;
    modes[2 * g.nx + m] = fac;
    modes[3 * g.nx + m] = tau;
}

// nu = sin(k_y) with sin^2(k_y/2) = k^2 eps/4 - sin^2(pi m/nx).
__device__ double nu_of(const GridDev &g, int m, double eps) {
    double sp = sinpi((double)m / (double)g.nx);
    double q = g.k * g.k * eps * 0.25 - sp * sp;
    double ky = 2.0 * asin(sqrt(q));
    return sin(ky);
}

__device__ __forceinline__ int mod_nx(int m, int nx) { int r = m % nx; return r < 0 ? r + nx : r; }

__global__ void k_channel_coef(GridDev g, const int *m_in, int n_in, const int *m_out, int n_out,
                               const double2 *modes, double2 *coef) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_in) {
        int m = m_in[c];
        double nu = nu_of(g, m, g.eps_sub);
        // source -2i sqrt(nu) carried to the first slab row
        double2 b = cmk(0.0, -2.0 * sqrt(nu));
        coef[c] = cmul(b, modes[2 * g.nx + mod_nx(m, g.nx)]);
    } else if (c < n_in + n_out) {
        int m = m_out[c - n_in];
        double nu = nu_of(g, m, g.eps_clad);
        coef[c] = cscale(modes[3 * g.nx + mod_nx(m, g.nx)], sqrt(nu));
    }
}

// Right-hand sides of the slab system (rows [row][col][x]):
// forward column a on the first slab row: beta_a u_{m_a}(x);
// adjoint column n_in+b on the last slab row: w_b u_{-m_b}(x)
// (C^T projected through the cladding; A = A^T).
__global__ void k_build_rhs(GridDev g, const int *m_in, int n_in, const int *m_out, int n_out,
                            const double2 *coef, double2 *E) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (x >= g.nx) return;
    int ncol = n_in + n_out;
    int row, m;
    if (c < n_in) { row = 0; m = m_in[c]; }
    else { row = g.h - 1; m = -m_out[c - n_in]; }
    long long t = ((long long)mod_nx(m, g.nx) * x) % g.nx;
    double sn, cs;
    sincospi(2.0 * (double)t / (double)g.nx, &sn, &cs);
    double inv = rsqrt((double)g.nx);
    double2 v = cmul(coef[c], cmk(cs * inv, sn * inv));
    E[((long long)row * ncol + c) * g.nx + x] = v;
}

// spec[a][(-m_b) mod nx] = Gamma[b][a] * w_b (output orders are distinct, so
// every (a, b) writes its own element).
__global__ void k_adjoint_spectrum(const double2 *Gamma, const double2 *coef, const int *m_out, int n_in, int n_out,
                                   int nx, double2 *spec) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    int b = blockIdx.y;
    if (a >= n_in) return;
    int m = mod_nx(-m_out[b], nx);
    spec[(long long)a * nx + m] = cmul(Gamma[(long long)b * n_in + a], coef[n_in + b]);
}

__global__ void k_twiddles(double2 *tw, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n / 2) return;
    double sn, cs;
    sincospi(-2.0 * (double)i / (double)n, &sn, &cs);
    tw[i] = cmk(cs, sn);
}

// Radix-2 decimation-in-time FFT of one length-n column per block, in shared
// memory: out[k] = scale * sum_x in[x] exp(sign * 2 pi i k x / n).
__global__ void k_fft(const double2 *in, double2 *out, int n, int logn, long long in_stride,
                      long long out_stride, int sign, double scale, const double2 *tw) {
    extern __shared__ double2 a[];
    const double2 *src = in + (long long)blockIdx.x * in_stride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        unsigned r = __brev((unsigned)i) >> (32 - logn);
        a[r] = src[i];
    }
    __syncthreads();
    for (int lh = 0; lh < logn; ++lh) {
        int half = 1 << lh;
        int tstride = n >> (lh + 1);
        for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
            int pos = t & (half - 1);
            int i = ((t >> lh) << (lh + 1)) + pos;
            int j = i + half;
            double2 w = tw[pos * tstride];
            if (sign > 0) w.y = -w.y;
            double2 u = a[i];
            double2 v = cmul(a[j], w);
            a[i] = cadd(u, v);
            a[j] = csub(u, v);
        }
        __syncthreads();
    }
    double2 *dst = out + (long long)blockIdx.x * out_stride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = cscale(a[i], scale);
}

// Source-row map of the substrate side, per Fourier order m: with the rows
// below the slab eliminated upward (pivots dt_j, couplings c_j = 1/s_{j-1/2}),
// back substitution gives the field on the source row as
//   u_src = fac[m] u_{j0} + q[m] b,
// u_{j0} the first slab row, b the source coefficient on the source row;
// fac is the boundary sweep's product of c_{i+1}/dt_i over i = src..j0-1 (A
// is symmetric, so the same factor carries the source up), and
// q = sum_{j=src}^{j0-1} G_j^2 / dt_j with G_src = 1, G_{j+1} = G_j c_{j+1}/dt_j.
__global__ void k_source_row(GridDev g, const double2 *st, double2 *q) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.nx) return;
    const double2 *ish = st + g.ny + 1;
    double sp = sinpi((double)m / (double)g.nx);
    double lam = 4.0 * sp * sp;
    double2 dt = row_diag(g, st, 0, lam, g.eps_sub);
    double2 G = cmk(1.0, 0.0), acc = cmk(0.0, 0.0);
    for (int j = 0; j < g.j0; ++j) {
        if (j > 0) dt = csub(row_diag(g, st, j, lam, g.eps_sub), cmul(cmul(ish[j], ish[j]), cinv(dt)));
        if (j >= g.jsrc) {
            const double2 idt = cinv(dt);
            acc = cadd(acc, cmul(cmul(G, G), idt));
            G = cmul(G, cmul(ish[j + 1], idt));
        }
    }
    q[m] = acc;
}

// Reflection block: R[b][a] = sqrt(nu_b) (fac[m_b] ehat_a[m_b] + [m_b == m_a] q[m_a] beta_a)
// - [m_b == m_a], beta_a = -2i sqrt(nu_a) the source coefficient of input a, ehat
// the (1/sqrt(nx)) FFT of forward column a on the first slab row.
__global__ void k_reflection(GridDev g, const double2 *fft0, const double2 *modes, const double2 *q,
                             const int *m_in, int n_in, const int *m_ref, int n_ref, double2 *R) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    int b = blockIdx.y;
    if (a >= n_in || b >= n_ref) return;
    const int mb = m_ref[b], ib = mod_nx(mb, g.nx);
    const double nub = nu_of(g, mb, g.eps_sub);
    double2 u = cmul(modes[2 * g.nx + ib], fft0[(long long)a * g.nx + ib]);
    const bool diag = (mb == m_in[a]);
    if (diag) u = cadd(u, cmul(q[ib], cmk(0.0, -2.0 * sqrt(nub))));
    double2 r = cscale(u, sqrt(nub));
    if (diag) r.x -= 1.0;
    R[(long long)b * n_in + a] = r;
}

// Transmission from the cladding side: adjoint column b solved A Phi_b = C_b^T,
// and a cladding source of order -m_b is -2i C_b^T, so the field it makes on
// the first slab row is -2i Phi_b.  Srev[p][qq] = sqrt(nu_p) fac[m_p] (-2i)
// phihat_{b}[m_p] with m_p = m_in[p] (substrate order) and b = rmap[qq] the
// adjoint column with m_out[b] = -m_out[qq] (cladding order m_out[qq]).
__global__ void k_reverse_S(GridDev g, const double2 *fft0, const double2 *modes, const int *m_in, int n_in,
                            const int *rmap, int n_out, double2 *Srev) {
    int qq = blockIdx.x * blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (qq >= n_out || p >= n_in) return;
    const int mp = m_in[p], ip = mod_nx(mp, g.nx);
    const double nup = nu_of(g, mp, g.eps_sub);
    const double2 phi = fft0[(long long)(n_in + rmap[qq]) * g.nx + ip];
    const double2 u = cmul(cmul(modes[2 * g.nx + ip], phi), cmk(0.0, -2.0));
    Srev[(long long)p * n_out + qq] = cscale(u, sqrt(nup));
}

}  // namespace

void launch_source_row(apf_ctx *c, double2 *q, cudaStream_t s) {
    GridDev g = make_grid(c);
    APF_LAUNCH(c, k_source_row, (c->nx + 127) / 128, 128, 0, s, g, c->d_stretch, q);
}

void launch_reflection(apf_ctx *c, const double2 *fft0, const double2 *q, const int *m_ref, int n_ref, double2 *R,
                       cudaStream_t s) {
    GridDev g = make_grid(c);
    dim3 grid((c->nin + 127) / 128, n_ref);
    APF_LAUNCH(c, k_reflection, grid, 128, 0, s, g, fft0, c->d_modes, q, c->d_min, c->nin, m_ref, n_ref, R);
}

void launch_reverse_S(apf_ctx *c, const double2 *fft0, const int *rmap, double2 *Srev, cudaStream_t s) {
    GridDev g = make_grid(c);
    dim3 grid((c->nout + 127) / 128, c->nin);
    APF_LAUNCH(c, k_reverse_S, grid, 128, 0, s, g, fft0, c->d_modes, c->d_min, c->nin, rmap, c->nout, Srev);
}

int fft_smem_bytes(int n) { return n * (int)sizeof(double2); }

void launch_twiddles(apf_ctx *c, cudaStream_t s) {
    int n = c->nx;
    APF_LAUNCH(c, k_twiddles, (n / 2 + 255) / 256, 256, 0, s, c->d_tw, n);
}

void launch_fft(apf_ctx *c, const double2 *in, double2 *out, int n, int batch, long long in_stride,
                long long out_stride, int sign, double scale, cudaStream_t s) {
    if (batch <= 0) return;
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    int smem = fft_smem_bytes(n);
    int threads = n / 2 < 256 ? n / 2 : 256;
    APF_LAUNCH(c, k_fft, batch, threads, smem, s, in, out, n, logn, in_stride, out_stride, sign, scale, c->d_tw);
}

void launch_boundary(apf_ctx *c, cudaStream_t s) {
    GridDev g = make_grid(c);
    APF_LAUNCH(c, k_stretch_table, (c->ny + 1 + 127) / 128, 128, 0, s, g, c->d_stretch);
    APF_LAUNCH(c, k_boundary_sweep, (c->nx + 63) / 64, 64, 0, s, g, c->d_stretch, c->d_modes);
    int nc = (c->nin + c->nout);
    APF_LAUNCH(c, k_channel_coef, (nc + 127) / 128, 128, 0, s, g, c->d_min, c->nin, c->d_mout,
               c->nout, c->d_modes, c->d_coef);
    // circulant generators: c(d) = (1/nx) sum_m sigma_m exp(2 pi i m d / nx)
    launch_fft(c, c->d_modes, c->d_circ, c->nx, 2, c->nx, c->nx, +1, 1.0 / c->nx, s);
}

void launch_build_rhs(apf_ctx *c, double2 *E, cudaStream_t s) {
    GridDev g = make_grid(c);
    // the columns of the current layout: cf forward (inputs), ca adjoint (outputs)
    int nf = c->cf, na = c->ca;
    dim3 grid((c->nx + 255) / 256, nf + na);
    APF_LAUNCH(c, k_build_rhs, grid, 256, 0, s, g, c->d_min, nf, c->d_mout, na, c->d_coef, E);
}

// Right-hand sides of the conventional adjoint method's second pass (Eq. S1):
// for input a, the adjoint source sum_b Gamma_ba C_b^T carried to the last slab
// row, i.e. sum_b Gamma_ba w_b u_{-m_b} (the adjoint column of output b is
// w_b u_{-m_b} on that row).  Written as a spectrum (order -m_b gets
// Gamma_ba w_b) and brought to pixels by one inverse FFT per column.
void launch_adjoint_rhs(apf_ctx *c, const double2 *Gamma, double2 *Erow, cudaStream_t s) {
    int nin = c->nin, nout = c->nout;
    launch_zero(c, c->d_fft, sizeof(double2) * (long long)nin * c->nx, s);
    dim3 grid((nin + 127) / 128, nout);
    APF_LAUNCH(c, k_adjoint_spectrum, grid, 128, 0, s, Gamma, c->d_coef, c->d_mout, nin, nout, c->nx, c->d_fft);
    launch_fft(c, c->d_fft, Erow, c->nx, nin, c->nx, c->nx, +1, 1.0 / sqrt((double)c->nx), s);
}

void boundary_init_attrs() {
    cudaFuncSetAttribute(k_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * (int)sizeof(double2));
}
