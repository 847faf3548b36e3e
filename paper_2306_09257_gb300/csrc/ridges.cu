// Ridge edge-position parametrization (paper Sec. 3, Eq. 5; mirror symmetry
// of the free half period, Supplement Sec. 7 without it): the slab
// permittivity of a ridge pattern and the chain rule from the pixel gradient
// to the edge positions.
#include "apf_internal.h"

#include <math.h>

namespace {

// One thread per pixel column: covered length of [x, x+1) (positions from the
// mirror plane x = nx/2), summed over the ridges and then their images; the
// same value on every slab row.
__global__ void k_ridge_eps(const double *__restrict__ e, int ne, int mirror, double eps_r, double eps_b, int nx,
                            int h, double *__restrict__ eps) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const double lo = (double)x - 0.5 * nx, hi = lo + 1.0;
    double fill = 0.0;
    for (int i = 0; i + 1 < ne; i += 2) fill += fmax(0.0, fmin(e[i + 1], hi) - fmax(e[i], lo));
    if (mirror)
        for (int i = 0; i + 1 < ne; i += 2) fill += fmax(0.0, fmin(-e[i], hi) - fmax(-e[i + 1], lo));
    const double v = eps_b + (eps_r - eps_b) * fill;
    for (int j = 0; j < h; ++j) eps[(long long)j * nx + x] = v;
}

__device__ __forceinline__ int wrap(long long p, int nx) { return (int)(((p % nx) + nx) % nx); }

// One warp per edge: the column sum of the pixel gradient under the pixel the
// edge moves into (and, with mirror symmetry, the one its image moves into),
// times -+(eps_r - eps_b).
__global__ void k_ridge_grad(const double *__restrict__ e, int ne, int mirror, double d_eps, int nx, int h,
                             const double *__restrict__ g, double *__restrict__ out) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= ne) return;
    const double t = e[k];
    const int px = wrap((long long)floor(t + 0.5 * nx), nx);
    const int pm = wrap((long long)ceil(0.5 * nx - t) - 1, nx);
    double sx = 0.0, sm = 0.0;
    for (int j = lane; j < h; j += 32) {
        sx += g[(long long)j * nx + px];
        if (mirror) sm += g[(long long)j * nx + pm];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, off);
        sm += __shfl_xor_sync(0xffffffffu, sm, off);
    }
    if (lane == 0) {
        const double sign = (k % 2 == 0) ? -1.0 : 1.0;
        out[k] = sign * d_eps * sx + (mirror ? sign * d_eps * sm : 0.0);
    }
}

int ensure_ridge_buffers(apf_ctx *c, int n_edges, long long n_eps) {
    if (n_edges > c->ridge_cap) {
        if (c->d_edges) cudaFree(c->d_edges);
        if (c->d_ridge_g) cudaFree(c->d_ridge_g);
        c->d_edges = c->d_ridge_g = nullptr;
        c->ridge_cap = 0;
        cudaError_t e = cudaMalloc(&c->d_edges, sizeof(double) * n_edges);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_ridge_g, sizeof(double) * n_edges);
        if (e != cudaSuccess) return check_cuda(c, e, "cudaMalloc ridge edges");
        c->ridge_cap = n_edges;
    }
    if (n_eps > c->ridge_eps_cap) {
        if (c->d_ridge_eps) cudaFree(c->d_ridge_eps);
        c->d_ridge_eps = nullptr;
        c->ridge_eps_cap = 0;
        cudaError_t e = cudaMalloc(&c->d_ridge_eps, sizeof(double) * n_eps);
        if (e != cudaSuccess) return check_cuda(c, e, "cudaMalloc ridge eps");
        c->ridge_eps_cap = n_eps;
    }
    return APF_OK;
}

}  // namespace

void ridges_free(apf_ctx *c) {
    if (c->d_edges) cudaFree(c->d_edges);
    if (c->d_ridge_g) cudaFree(c->d_ridge_g);
    if (c->d_ridge_eps) cudaFree(c->d_ridge_eps);
    c->d_edges = c->d_ridge_g = c->d_ridge_eps = nullptr;
    c->ridge_cap = 0;
    c->ridge_eps_cap = 0;
    c->ridge_n = 0;
}

extern "C" {

int apf_set_ridges(apf_ctx *c, const double *edges, int n_edges, int mirror, double eps_ridge, double eps_bg,
                   int j0, int h, double eps_sub, double eps_clad, double *eps_out, void *stream) {
    if (!c) return APF_EINVAL;
    if (!c->grid_set) return set_err(c, APF_ESTATE, "apf_set_ridges before apf_set_grid");
    if (!edges) return set_err(c, APF_EINVAL, "edges is NULL");
    if (n_edges < 2 || (n_edges & 1)) return set_err(c, APF_EINVAL, "n_edges=%d must be even and >= 2", n_edges);
    if (h < 1) return set_err(c, APF_EINVAL, "h=%d must be >= 1", h);
    if (!(eps_ridge > 0.0) || !(eps_bg > 0.0) || !isfinite(eps_ridge) || !isfinite(eps_bg))
        return set_err(c, APF_EINVAL, "ridge and background permittivities must be positive and finite");
    cudaSetDevice(c->device);
    std::vector<double> t(n_edges);
    cudaStream_t caller = (cudaStream_t)stream;
    if (is_device_ptr(edges)) {
        // device edges are read in order on the caller's stream, after the work that produced them
        cudaError_t e = cudaMemcpyAsync(t.data(), edges, sizeof(double) * n_edges, cudaMemcpyDeviceToHost, caller);
        if (e == cudaSuccess) e = cudaStreamSynchronize(caller);
        if (e != cudaSuccess) return check_cuda(c, e, "read edges");
    } else {
        for (int i = 0; i < n_edges; ++i) t[i] = edges[i];
    }
    const double lo = -0.5 * c->nx, hi = mirror ? 0.0 : 0.5 * c->nx;
    for (int i = 0; i < n_edges; ++i) {
        if (!isfinite(t[i])) return set_err(c, APF_EINVAL, "edge %d is not finite", i);
        if (t[i] < lo || t[i] > hi) return set_err(c, APF_EINVAL, "edge %d = %g outside [%g, %g]", i, t[i], lo, hi);
        if (i > 0 && t[i] < t[i - 1]) return set_err(c, APF_EINVAL, "edges not sorted at %d", i);
    }
    long long n = (long long)h * c->nx;
    int rc = ensure_ridge_buffers(c, n_edges, n);
    if (rc) return rc;
    cudaStream_t s = c->cap_stream;
    cudaError_t e = cudaMemcpyAsync(c->d_edges, t.data(), sizeof(double) * n_edges, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return check_cuda(c, e, "upload edges");
    APF_LAUNCH(c, k_ridge_eps, (c->nx + 127) / 128, 128, 0, s, c->d_edges, n_edges, mirror ? 1 : 0, eps_ridge,
               eps_bg, c->nx, h, c->d_ridge_eps);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(c, e, "ridge eps");
    c->ridge_n = n_edges;
    c->ridge_h = h;
    c->ridge_mirror = mirror ? 1 : 0;
    c->ridge_eps_r = eps_ridge;
    c->ridge_eps_b = eps_bg;
    // the generated slab was written (and synchronized) on the context's own stream
    rc = apf_set_eps(c, c->d_ridge_eps, j0, h, eps_sub, eps_clad, (void *)s);
    if (rc) return rc;
    if (eps_out) {
        // written in order on the caller's stream (after its earlier work on eps_out)
        e = cudaMemcpyAsync(eps_out, c->d_ridge_eps, sizeof(double) * n, cudaMemcpyDefault, caller);
        if (e == cudaSuccess) e = cudaStreamSynchronize(caller);
        if (e != cudaSuccess) return check_cuda(c, e, "eps_out");
    }
    return APF_OK;
}

int apf_ridge_grad(apf_ctx *c, const double *grad_eps, double *grad_edges, void *stream) {
    if (!c) return APF_EINVAL;
    if (!grad_eps || !grad_edges) return set_err(c, APF_EINVAL, "grad_eps / grad_edges is NULL");
    if (c->ridge_n <= 0) return set_err(c, APF_ESTATE, "apf_ridge_grad needs apf_set_ridges first");
    if (c->ridge_h != c->h) return set_err(c, APF_ESTATE, "the slab changed since apf_set_ridges");
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)c->ridge_h * c->nx;
    const double *g = grad_eps;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(grad_eps)) {
        // the generated eps has been copied into the solver; its buffer stages the host gradient
        e = cudaMemcpyAsync(c->d_ridge_eps, grad_eps, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return check_cuda(c, e, "upload grad_eps");
        g = c->d_ridge_eps;
    }
    const bool dev_out = is_device_ptr(grad_edges);
    double *out = dev_out ? grad_edges : c->d_ridge_g;
    APF_LAUNCH(c, k_ridge_grad, (c->ridge_n + 7) / 8, 256, 0, s, c->d_edges, c->ridge_n, c->ridge_mirror,
               c->ridge_eps_r - c->ridge_eps_b, c->nx, c->ridge_h, g, out);
    if (!dev_out) e = cudaMemcpyAsync(grad_edges, out, sizeof(double) * c->ridge_n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(c, e, "ridge grad");
    return APF_OK;
}

}  // extern "C"
