// Allocation-free small-grid solve: the same float64 pipeline as
// apf_solve_S (boundary sweep, slab elimination, field sweeps, FFT readout),
// with every intermediate array carved out of one file-scope device array
// instead of cudaMalloc'd workspace.
#include "apf_internal.h"

#include <math.h>
#include <string.h>

namespace {

constexpr size_t kScratchBytes = APF_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxNx = 64, kMaxH = 16, kMaxCols = 128;

// One copy per GPU that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once (host code may not
// use the symbol itself as a device pointer).
void *g_scratch_dev[64] = {nullptr};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int fail(int code, const char *msg) { return set_err(nullptr, code, "apf_solve_S_noalloc: %s", msg); }

double disp_q(int nx, double k, int m, double eps) {
    double s = sin(M_PI * (double)m / (double)nx);
    return k * k * eps / 4.0 - s * s;
}

}  // namespace

extern "C" int apf_solve_S_noalloc(int nx, int ny, int npml_bot, int npml_top, double lambda_px,
                                   const apf_pml_params *pml, const double *eps_slab, int j0, int h,
                                   double eps_sub, double eps_clad, const int *m_in, int n_in, const int *m_out,
                                   int n_out, double *S, void *stream) {
    // ---- argument checks (host, before any launch) ----
    if (nx < 8 || nx > kMaxNx || (nx & (nx - 1))) return fail(APF_EINVAL, "nx must be a power of two in [8, 64]");
    if (h < 1 || h > kMaxH) return fail(APF_EINVAL, "h must be in [1, 16]");
    if (npml_bot < 1 || npml_top < 1 || ny < npml_bot + npml_top + 4 || ny > 4096)
        return fail(APF_EINVAL, "bad PML / ny (ny <= 4096)");
    if (!(lambda_px > 2.0) || !isfinite(lambda_px)) return fail(APF_EINVAL, "lambda_px must be > 2");
    if (!eps_slab || !S) return fail(APF_EINVAL, "eps_slab and S must not be NULL");
    if (!(eps_sub > 0.0 && eps_clad > 0.0 && eps_clad <= eps_sub && isfinite(eps_sub)))
        return fail(APF_EINVAL, "need 0 < eps_clad <= eps_sub, finite");
    double R0 = pml ? pml->R0 : 1e-8, power = pml ? pml->power : 3.0;
    if (!(R0 > 0.0 && R0 < 1.0) || !(power >= 0.0 && power <= 10.0)) return fail(APF_EINVAL, "bad PML parameters");
    if (j0 < 0) j0 = npml_bot + (ny - npml_bot - npml_top - h) / 2;
    int jsrc = npml_bot, jout = ny - npml_top - 1;
    if (!(jsrc < j0 && j0 + h <= jout)) return fail(APF_EINVAL, "slab must lie between the source and output rows");
    double k = 2.0 * M_PI / lambda_px;
    int ords_in[kMaxCols], ords_out[kMaxCols], nall = 0, all[kMaxNx];
    for (int m = -(nx / 2); m < nx - nx / 2; ++m) {
        double q = disp_q(nx, k, m, eps_clad);
        if (q > 0.0 && q < 1.0) all[nall++] = m;
    }
    if (!m_in || n_in <= 0) { n_in = nall; m_in = all; }
    if (!m_out || n_out <= 0) { n_out = nall; m_out = all; }
    if (n_in < 1 || n_out < 1 || n_in + n_out > kMaxCols) return fail(APF_EINVAL, "need 1..128 channels in total");
    for (int a = 0; a < n_in; ++a) {
        double q = disp_q(nx, k, m_in[a], eps_sub);
        if (!(q > 0.0 && q < 1.0)) return fail(APF_EINVAL, "an input order does not propagate in the substrate");
        ords_in[a] = m_in[a];
    }
    for (int b = 0; b < n_out; ++b) {
        double q = disp_q(nx, k, m_out[b], eps_clad);
        if (!(q > 0.0 && q < 1.0)) return fail(APF_EINVAL, "an output order does not propagate in the cladding");
        if (b > 0 && m_out[b] <= m_out[b - 1]) return fail(APF_EINVAL, "output orders must be strictly ascending");
        ords_out[b] = m_out[b];
    }
    cudaStream_t s = (cudaStream_t)stream;
    {
        // the permittivity must be finite (checked on the host, from a stack copy if it is on the device;
        // the copy is read in order on the caller's stream, after the work that produced eps_slab)
        double tmp[kMaxH * kMaxNx];
        cudaPointerAttributes at;
        bool on_dev = cudaPointerGetAttributes(&at, eps_slab) == cudaSuccess &&
                      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        const double *src = eps_slab;
        if (on_dev) {
            cudaError_t e = cudaMemcpyAsync(tmp, eps_slab, sizeof(double) * h * nx, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return set_err(nullptr, APF_ECUDA, "apf_solve_S_noalloc: cannot read eps_slab: %s",
                               cudaGetErrorString(e));
            }
            src = tmp;
        }
        for (int i = 0; i < h * nx; ++i)
            if (!isfinite(src[i])) return fail(APF_EINVAL, "eps_slab is not finite");
    }
    // ---- the scratch array of the current device ----
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(APF_ECUDA, "no current CUDA device");
    }
    // one call at a time per device (with every other solve of the library),
    // so overlapping calls from several threads never share the scratch array
    SolveGate gate(dev);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_err(nullptr, APF_ECUDA, "apf_solve_S_noalloc: cudaGetSymbolAddress failed: %s",
                           cudaGetErrorString(e));
        }
        g_scratch_dev[dev] = p;
    }
    unsigned char *base = (unsigned char *)g_scratch_dev[dev];
    const long long n = nx, ncol = n_in + n_out;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += align256(bytes);
        return (void *)p;
    };
    // ---- a host-side context whose device pointers all point into g_scratch ----
    apf_ctx c;
    c.device = dev;
    c.precision = APF_FP64;
    c.nx = nx; c.ny = ny; c.npml_bot = npml_bot; c.npml_top = npml_top;
    c.lambda_px = lambda_px; c.k = k; c.R0 = R0; c.power = power;
    c.h = h; c.j0 = j0; c.eps_sub = eps_sub; c.eps_clad = eps_clad;
    c.nin = n_in; c.nout = n_out;
    c.grid_set = c.eps_set = c.ch_set = true;
    c.use_graphs = false;
    c.d_eps = (double *)carve(sizeof(double) * h * n);
    c.d_min = (int *)carve(sizeof(int) * kMaxCols);
    c.d_mout = (int *)carve(sizeof(int) * kMaxCols);
    c.d_modes = (double2 *)carve(sizeof(double2) * 4 * n);
    c.d_stretch = (double2 *)carve(sizeof(double2) * 2 * (ny + 1));
    c.d_coef = (double2 *)carve(sizeof(double2) * ncol);
    c.d_circ = (double2 *)carve(sizeof(double2) * 2 * n);
    c.d_tw = (double2 *)carve(sizeof(double2) * n / 2);
    c.d_G = (double2 *)carve(sizeof(double2) * h * n * n);
    c.d_scr1 = (double2 *)carve(sizeof(double2) * n * n / 2);
    c.d_scr2 = (double2 *)carve(sizeof(double2) * n * n / 2);
    c.d_E = (double2 *)carve(sizeof(double2) * h * ncol * n);
    c.d_T = (double2 *)carve(sizeof(double2) * ncol * n);
    c.d_fft = (double2 *)carve(sizeof(double2) * ncol * n);
    c.d_S = (double2 *)carve(sizeof(double2) * n_in * n_out);
    c.d_flags = (int *)carve(sizeof(int) * 4);
    if (off > kScratchBytes) return fail(APF_EINVAL, "problem does not fit the scratch array");
    // one sweep of all forward and adjoint columns, as in apf_solve_S
    c.lay = 0; c.cf = n_in; c.ca = n_out; c.d_Ew = c.d_E;
    // ---- the pipeline (same kernels as apf_solve_S in APF_FP64) ----
    cudaError_t ce = cudaMemcpyAsync(c.d_eps, eps_slab, sizeof(double) * h * n, cudaMemcpyDefault, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(c.d_min, ords_in, sizeof(int) * n_in, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(c.d_mout, ords_out, sizeof(int) * n_out, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c.d_flags, 0, 4 * sizeof(int), s);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return set_err(nullptr, APF_ECUDA, "apf_solve_S_noalloc: upload: %s", cudaGetErrorString(ce));
    }
    launch_twiddles(&c, s);
    launch_boundary(&c, s);
    for (int j = 0; j < h; ++j) {
        double2 *X = c.d_G + (long long)j * n * n;
        launch_assemble64(&c, j, X, j > 0 ? c.d_G + (long long)(j - 1) * n * n : nullptr, s);
        invert_sym64(&c, X, nx, n, c.d_scr1, c.d_scr2, s);
    }
    launch_zero(&c, c.d_E, sizeof(double2) * h * ncol * n, s);  // the fields must start at zero
    launch_build_rhs(&c, c.d_E, s);
    fields64(&c, s);
    launch_readout(&c, s);
    // a failed launch (configuration or resources) is reported here, before the
    // sync, so that S is never taken from an earlier call's leftovers
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        cudaStreamSynchronize(s);
        return set_err(nullptr, APF_ECUDA, "apf_solve_S_noalloc: kernel launch: %s", cudaGetErrorString(ce));
    }
    ce = cudaMemcpyAsync(S, c.d_S, sizeof(double2) * n_in * n_out, cudaMemcpyDefault, s);
    int flags = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&flags, c.d_flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = ce;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(nullptr, APF_ECUDA, "apf_solve_S_noalloc: %s", cudaGetErrorString(e));
    }
    if (flags & FLAG_SINGULAR) return fail(APF_ESINGULAR, "zero pivot in a diagonal-block inversion");
    if (flags & FLAG_TIMEOUT) return fail(APF_ETIMEOUT, "a bounded device wait gave up");
    if (flags & FLAG_NONFINITE) return fail(APF_ECUDA, "non-finite value in the elimination");
    return APF_OK;
}
