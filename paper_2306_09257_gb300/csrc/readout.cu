// S readout, objective f with its Wirtinger derivative Gamma = df/dS, and the
// adjoint contraction for the permittivity gradient.
#include "apf_internal.h"

namespace {

__device__ __forceinline__ int mod_n(int m, int n) { int r = m % n; return r < 0 ? r + n : r; }

// S[b][a] = w_b * ehat_a[m_b], ehat = (1/sqrt(nx)) FFT of the forward field
// on the last slab row (the projection C_b carried through the cladding).
__global__ void k_gather_S(const double2 *fft, const double2 *coef, const int *m_out, int n_in, int n_out,
                           int nx, double2 *S) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    int b = blockIdx.y;
    if (a >= n_in) return;
    int m = mod_n(m_out[b], nx);
    S[(long long)b * n_in + a] = cmul(coef[n_in + b], fft[(long long)a * nx + m]);
}

struct Orders {
    int n;
    int d[16];
};

// One thread per (input a, relative order d): output b with m_out[b] = m_in[a]+d
// (binary search over the ascending m_out).  kind 1: f = sum |S|^2,
// Gamma = conj(S).  kind 2: f = sum (|S|^2 - t)^2, Gamma = 2(|S|^2 - t) conj(S)
// (Eq. 5 and the derivative printed after it).  f is reduced in a fixed order.
__global__ void k_objective(const double2 *S, const int *m_in, const int *m_out, int n_in, int n_out,
                            Orders ord, int kind, double t, double2 *Gam, double *f_out) {
    __shared__ double red[1024];
    double acc = 0.0;
    int total = n_in * ord.n;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int a = e / ord.n, di = e - a * ord.n;
        int target = m_in[a] + ord.d[di];
        int lo = 0, hi = n_out - 1, b = -1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int v = m_out[mid];
            if (v == target) { b = mid; break; }
            if (v < target) lo = mid + 1; else hi = mid - 1;
        }
        if (b < 0) continue;
        double2 s = S[(long long)b * n_in + a];
        double p = cabs2(s);
        double2 g;
        if (kind == APF_OBJ_POWER) {
            acc += p;
            g = cconj(s);
        } else {
            acc += (p - t) * (p - t);
            g = cscale(cconj(s), 2.0 * (p - t));
        }
        Gam[(long long)b * n_in + a] = g;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) f_out[0] = red[0];
}

// g[j][x] = 2 k^2 Re sum_b Phi_j[b][x] Q_j[b][x], with Q_j = Gamma F_j.
// This is Eq. (1) with Eq. (3): dS_ba/deps_k = k^2 (C A^-1)_{b,k} (A^-1 B)_{k,a}
// and (C A^-1)_{b,k} = (A^-1 C^T)_{k,b} = Phi_{k,b} because A = A^T.
__global__ void k_grad_rowdot(const double2 *E, const double2 *Q, int h, int nx, int n_in, int n_out,
                              double k2, double *g) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (x >= nx) return;
    int ncol = n_in + n_out;
    const double2 *phi = E + ((long long)j * ncol + n_in) * nx + x;
    const double2 *q = Q + (long long)j * n_out * nx + x;
    double acc = 0.0;
    for (int b = 0; b < n_out; ++b) {
        double2 p = phi[(long long)b * nx], qq = q[(long long)b * nx];
        acc += p.x * qq.x - p.y * qq.y;
    }
    g[(long long)j * nx + x] = 2.0 * k2 * acc;
}

// Conventional adjoint method (Eq. S1): g[j][x] = 2 k^2 Re sum_a lam_a[j][x] F_a[j][x],
// with the forward fields F_a = A^-1 B_a and the adjoint fields
// lam_a = A^-1 (C_a^adj)^T, C_a^adj = sum_b Gamma_ba C_b, both [row][a][x]
// with n_in columns.  One thread per pixel, the sum over a in a fixed order.
__global__ void k_grad_adjoint(const double2 *F, const double2 *Lam, int h, int nx, int n_in, double k2, double *g) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (x >= nx) return;
    const long long o = (long long)j * n_in * nx + x;
    double acc = 0.0;
    for (int a = 0; a < n_in; ++a) {
        const double2 f = F[o + (long long)a * nx], l = Lam[o + (long long)a * nx];
        acc = fma(f.x, l.x, acc);
        acc = fma(-f.y, l.y, acc);
    }
    g[(long long)j * nx + x] = 2.0 * k2 * acc;
}

}  // namespace

void launch_gradient_adjoint(apf_ctx *c, const double2 *Fw, const double2 *Lam, cudaStream_t s) {
    dim3 grid((c->nx + 255) / 256, c->h);
    APF_LAUNCH(c, k_grad_adjoint, grid, 256, 0, s, Fw, Lam, c->h, c->nx, c->nin, c->k * c->k, c->d_grad);
}

void launch_readout(apf_ctx *c, cudaStream_t s) {
    // forward columns come first in every layout that carries them (cf = n_in)
    int nin = c->nin, nout = c->nout, ncol = c->cf + c->ca;
    const double2 *Eh = c->d_Ew + (long long)(c->h - 1) * ncol * c->nx;
    launch_fft(c, Eh, c->d_fft, c->nx, nin, c->nx, c->nx, -1, 1.0 / sqrt((double)c->nx), s);
    dim3 grid((nin + 127) / 128, nout);
    APF_LAUNCH(c, k_gather_S, grid, 128, 0, s, c->d_fft, c->d_coef, c->d_mout, nin, nout, c->nx, c->d_S);
}

int launch_objective(apf_ctx *c, int objective, const double *params, int n_params, cudaStream_t s) {
    if (objective != APF_OBJ_POWER && objective != APF_OBJ_SPLITTER)
        return set_err(c, APF_EINVAL, "unknown objective id %d", objective);
    if (!params || n_params < 2) return set_err(c, APF_EINVAL, "objective params need {t, nD, d...}");
    int nd = (int)params[1];
    if (nd < 1 || nd > 16 || n_params != 2 + nd)
        return set_err(c, APF_EINVAL, "objective: nD=%d must be in [1,16] and n_params = 2+nD", nd);
    Orders o{};
    o.n = nd;
    for (int i = 0; i < nd; ++i) {
        double v = params[2 + i];
        if (v != (double)(int)v) return set_err(c, APF_EINVAL, "objective order %g is not an integer", v);
        o.d[i] = (int)v;
    }
    int nin = c->nin, nout = c->nout;
    cudaMemsetAsync(c->d_Gam, 0, sizeof(double2) * (size_t)nin * nout, s);
    APF_LAUNCH(c, k_objective, 1, 1024, 0, s, c->d_S, c->d_min, c->d_mout, nin, nout, o, objective, params[0],
               c->d_Gam, c->d_f);
    return APF_OK;
}

int launch_gradient(apf_ctx *c, const double2 *Gamma, cudaStream_t s) {
    if (c->precision != APF_FP64) return mixed_gradient(c, Gamma, s);
    int nin = c->nin, nout = c->nout, ncol = nin + nout;
    long long nx = c->nx;
    // Q_j = Gamma (n_out x n_in) * F_j (n_in x nx), batched over the slab rows
    zgemm(c, false, false, nout, c->nx, nin, cmk(1, 0), Gamma, nin, 0, c->d_E, nx, (long long)ncol * nx, cmk(0, 0),
          c->d_Q, nx, (long long)nout * nx, c->h, s);
    dim3 grid((c->nx + 255) / 256, c->h);
    APF_LAUNCH(c, k_grad_rowdot, grid, 256, 0, s, c->d_E, c->d_Q, c->h, c->nx, nin, nout, c->k * c->k, c->d_grad);
    return APF_OK;
}
