// C ABI of libapf: argument checks, workspace, and the solve pipeline.
//
// One solve = (a2) per-mode boundary elimination -> (a3/a4) slab assembly and
// block-Schur elimination -> (a5/a6) right-hand-side sweeps for the M_in
// forward and M_out adjoint columns (+ refinement in mixed mode) -> (a7) S,
// f, Gamma -> (a8) adjoint contraction.  These are the single-elimination
// counterparts of the paper's APF with the augmented inputs B~ = [B, U] and
// outputs C~ = [C; U^T] (Eq. 4): the slab fields F = (A^-1 B)|slab = U^T A^-1 B
// and Phi = (A^-1 C^T)|slab = (C A^-1 U)^T are exactly the two blocks the
// gradient needs, and U^T A^-1 U is never formed.
#include "apf_internal.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <mutex>


static char g_create_err[512] = "no error";

// Why one: with several solves in flight on separate streams of one GPU
// (three or four batched calls; sixteen single-design calls; once in ten
// runs two batched calls), a tensor-core launch on GB300 stayed resident
// without progress (GPU busy at idle power, no kernel fault, the GPU usable
// again once the process ended; the cause was not found), while one solve at
// a time never did.  So solve calls on one device run one at a time.
namespace {
constexpr int GATE_DEVICES = 64;
std::mutex g_gate_mu;
std::condition_variable g_gate_cv;
int g_gate_busy[GATE_DEVICES] = {}, g_gate_peak = 0;
thread_local int t_gate_depth = 0;
}  // namespace

SolveGate::SolveGate(int device)
    : dev_(device < 0 ? 0 : device % GATE_DEVICES), held_(t_gate_depth++ == 0) {
    if (!held_) return;
    std::unique_lock<std::mutex> lk(g_gate_mu);
    g_gate_cv.wait(lk, [this] { return g_gate_busy[dev_] == 0; });
    g_gate_peak = std::max(g_gate_peak, ++g_gate_busy[dev_]);
}

SolveGate::~SolveGate() {
    --t_gate_depth;
    if (!held_) return;
    {
        std::lock_guard<std::mutex> lk(g_gate_mu);
        --g_gate_busy[dev_];
    }
    g_gate_cv.notify_all();
}

// Test hook: the most solve calls seen inside the gate of one device at once (reset to 0 if asked).
extern "C" int apf_debug_inflight_peak(int reset) {
    std::lock_guard<std::mutex> lk(g_gate_mu);
    const int p = g_gate_peak;
    if (reset) g_gate_peak = 0;
    return p;
}



int set_err(apf_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else memcpy(g_create_err, buf, sizeof g_create_err);
    return code;
}

int check_cuda(apf_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return APF_OK;
    cudaGetLastError();
    return set_err(c, e == cudaErrorMemoryAllocation ? APF_ENOMEM : APF_ECUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

GridDev make_grid(const apf_ctx *c) {
    GridDev g;
    g.nx = c->nx; g.ny = c->ny; g.npml_bot = c->npml_bot; g.npml_top = c->npml_top;
    g.j0 = c->j0; g.h = c->h; g.jsrc = c->npml_bot; g.jout = c->ny - c->npml_top - 1;
    g.k = c->k; g.eps_sub = c->eps_sub; g.eps_clad = c->eps_clad; g.R0 = c->R0; g.power = c->power;
    return g;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void free_workspace(apf_ctx *c) {
    graphs_reset(c);
    mixed_free(c);
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->ws_bytes = 0;
    c->ws_nx = c->ws_ny = c->ws_h = c->ws_min = c->ws_mout = -1;
    c->d_min = c->d_mout = nullptr; c->d_stretch = nullptr; c->d_modes = c->d_coef = c->d_circ = c->d_tw = nullptr;
    c->d_G = c->d_scr1 = c->d_scr2 = c->d_E = c->d_T = c->d_R = nullptr;
    c->d_S = c->d_Gam = c->d_Q = c->d_fft = nullptr;
    c->d_grad = c->d_f = c->d_colnorm = nullptr;
    c->d_flags = nullptr; c->d_pairs = nullptr;
    c->d_qsrc = c->d_refl = c->d_srev = nullptr;
    c->d_mref = c->d_rmap = nullptr;
}

template <typename T>
static int dalloc(apf_ctx *c, T **p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, APF_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    c->ws_bytes += (long long)bytes;
    *p = (T *)q;
    return APF_OK;
}

// (Re)allocate the solve workspace when the problem size changed.  Solves never allocate.
static int ensure_workspace(apf_ctx *c) {
    int nin = c->nin, nout = c->nout;
    if (c->ws_nx == c->nx && c->ws_ny == c->ny && c->ws_h == c->h && c->ws_min == nin && c->ws_mout == nout)
        return APF_OK;
    free_workspace(c);
    long long nx = c->nx, h = c->h, ncol = nin + nout;
    int rc;
#define AL(p, n) if ((rc = dalloc(c, &(p), (size_t)(n))) != APF_OK) { free_workspace(c); return rc; }
    AL(c->d_min, nin); AL(c->d_mout, nout);
    AL(c->d_modes, 4 * nx); AL(c->d_stretch, 2 * (c->ny + 1)); AL(c->d_coef, ncol); AL(c->d_circ, 2 * nx); AL(c->d_tw, nx / 2);
    if (c->precision == APF_FP64) {
        AL(c->d_G, h * nx * nx);
        AL(c->d_scr1, nx * nx / 2); AL(c->d_scr2, nx * nx / 2);
    }
    // fields: the single-elimination solve's n_in + n_out columns, or the
    // conventional adjoint method's n_in forward and n_in adjoint columns
    AL(c->d_E, h * std::max<long long>(ncol, 2LL * nin) * nx); AL(c->d_T, ncol * nx); AL(c->d_fft, ncol * nx);
    if (c->precision != APF_FP64) { AL(c->d_R, h * ncol * nx); }
    AL(c->d_S, (long long)nout * nin); AL(c->d_Gam, (long long)nout * nin);
    AL(c->d_Q, h * nout * nx); AL(c->d_grad, h * nx);
    AL(c->d_f, 8); AL(c->d_colnorm, 2 * ncol); AL(c->d_flags, 4);
    AL(c->d_qsrc, nx); AL(c->d_refl, nx * nin); AL(c->d_srev, (long long)nin * nout);
    AL(c->d_mref, nx); AL(c->d_rmap, nout);
#undef AL
    if (c->precision != APF_FP64) {
        if ((rc = mixed_alloc(c)) != APF_OK) { free_workspace(c); return rc; }
    }
    // set-up work runs on the context's own non-blocking stream (never the legacy
    // stream or a device-wide sync, which other threads' graph captures forbid)
    cudaStream_t ss = c->cap_stream;
    cudaError_t e = cudaMemcpyAsync(c->d_min, c->m_in.data(), sizeof(int) * nin, cudaMemcpyHostToDevice, ss);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mout, c->m_out.data(), sizeof(int) * nout, cudaMemcpyHostToDevice, ss);
    if (e != cudaSuccess) { free_workspace(c); return check_cuda(c, e, "upload channels"); }
    launch_twiddles(c, ss);
    e = cudaStreamSynchronize(ss);
    if (e != cudaSuccess) { free_workspace(c); return check_cuda(c, e, "twiddles"); }
    c->ws_nx = c->nx; c->ws_ny = c->ny; c->ws_h = c->h; c->ws_min = nin; c->ws_mout = nout;
    return APF_OK;
}

// ---------------------------------------------------------------------------
// Channel selection: orders propagating in a uniform medium of the grid
// (5-point dispersion sin^2(k_y/2) = k^2 eps/4 - sin^2(pi m/nx) in (0, 1)).
// ---------------------------------------------------------------------------
static double disp_q(const apf_ctx *c, int m, double eps) {
    double s = sin(M_PI * (double)m / (double)c->nx);
    return c->k * c->k * eps / 4.0 - s * s;
}

extern "C" {

int apf_version(void) { return (2 << 16) | 0; }

int apf_create(apf_ctx **out, int cuda_device, int precision) {
    if (!out) return set_err(nullptr, APF_EINVAL, "apf_create: out is NULL");
    *out = nullptr;
    if (precision == APF_MIXED_TF32)
        return set_err(nullptr, APF_EINVAL, "apf_create: APF_MIXED_TF32 is reserved (not built); use APF_MIXED_BF16X3");
    if (precision != APF_FP64 && precision != APF_MIXED_BF16X3)
        return set_err(nullptr, APF_EINVAL, "apf_create: unknown precision %d", precision);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_err(nullptr, APF_ECUDA, "apf_create: no CUDA device (%s)", cudaGetErrorString(e));
    }
    if (cuda_device < 0 || cuda_device >= ndev)
        return set_err(nullptr, APF_EINVAL, "apf_create: device %d not in [0,%d)", cuda_device, ndev);
    e = cudaSetDevice(cuda_device);
    if (e != cudaSuccess) return set_err(nullptr, APF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    if (precision == APF_MIXED_BF16X3) {
        cudaDeviceProp p;
        cudaGetDeviceProperties(&p, cuda_device);
        if (p.major != 10 || p.minor != 3)
            return set_err(nullptr, APF_EINVAL, "mixed mode needs an sm_103 GPU (found sm_%d%d)", p.major, p.minor);
    }
    apf_ctx *c = new apf_ctx();
    c->device = cuda_device;
    c->precision = precision;
    c->butterfly = precision == APF_MIXED_BF16X3 ? 1 : 0;  // see apf_set_elimination
    if (const char *e = getenv("APF_GRAPHS")) c->use_graphs = e[0] != '0';  // diagnostic knob: 0 = launch eagerly
    for (auto &ev : c->ev) cudaEventCreate(&ev);
    cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    slab64_init_attrs();
    boundary_init_attrs();
    mixed_init_attrs();
    if (precision != APF_FP64 && tc_init() != APF_OK) {
        apf_destroy(c);
        return set_err(nullptr, APF_ECUDA, "cuTensorMapEncodeTiled unavailable from the driver");
    }
    *out = c;
    return APF_OK;
}

void apf_destroy(apf_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->cap_stream) cudaStreamSynchronize(c->cap_stream);
    free_workspace(c);
    if (c->d_eps) cudaFree(c->d_eps);
    ridges_free(c);
    for (auto &ev : c->ev) if (ev) cudaEventDestroy(ev);
    for (auto &ev : c->prof_ev) if (ev) cudaEventDestroy(ev);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char *apf_last_error(const apf_ctx *c) { return c ? c->err.c_str() : g_create_err; }

int apf_set_grid(apf_ctx *c, int nx, int ny, int npml_bot, int npml_top, double lambda_px,
                 const apf_pml_params *pml) {
    if (!c) return APF_EINVAL;
    if (nx < 8 || nx > 8192 || (nx & (nx - 1)))
        return set_err(c, APF_EINVAL, "nx=%d must be a power of two in [8, 8192]", nx);
    if (npml_bot < 1 || npml_top < 1) return set_err(c, APF_EINVAL, "PML thickness must be >= 1");
    if (ny < npml_bot + npml_top + 4) return set_err(c, APF_EINVAL, "ny=%d too small for the PMLs", ny);
    if (!(lambda_px > 2.0) || !isfinite(lambda_px)) return set_err(c, APF_EINVAL, "lambda_px must be > 2");
    double R0 = 1e-8, power = 3.0;
    if (pml) { R0 = pml->R0; power = pml->power; }
    if (!(R0 > 0.0 && R0 < 1.0) || !(power >= 0.0 && power <= 10.0))
        return set_err(c, APF_EINVAL, "PML parameters out of range (0<R0<1, 0<=p<=10)");
    c->nx = nx; c->ny = ny; c->npml_bot = npml_bot; c->npml_top = npml_top;
    c->lambda_px = lambda_px; c->k = 2.0 * M_PI / lambda_px; c->R0 = R0; c->power = power;
    c->grid_set = true;
    c->eps_set = false;
    c->ch_set = false;
    graphs_reset(c);
    return APF_OK;
}

int apf_set_eps(apf_ctx *c, const double *eps_slab, int j0, int h, double eps_sub, double eps_clad, void *stream) {
    if (!c) return APF_EINVAL;
    if (!c->grid_set) return set_err(c, APF_ESTATE, "apf_set_eps before apf_set_grid");
    if (!eps_slab) return set_err(c, APF_EINVAL, "eps_slab is NULL");
    if (h < 1) return set_err(c, APF_EINVAL, "h=%d must be >= 1", h);
    int jsrc = c->npml_bot, jout = c->ny - c->npml_top - 1;
    if (j0 < 0) j0 = c->npml_bot + (c->ny - c->npml_bot - c->npml_top - h) / 2;
    if (!(jsrc < j0 && j0 + h <= jout))
        return set_err(c, APF_EINVAL, "slab rows [%d,%d) must lie strictly between source row %d and output row %d",
                       j0, j0 + h, jsrc, jout);
    if (!(eps_sub > 0.0) || !(eps_clad > 0.0) || !isfinite(eps_sub) || !isfinite(eps_clad))
        return set_err(c, APF_EINVAL, "background permittivities must be positive and finite");
    if (eps_clad > eps_sub) return set_err(c, APF_EINVAL, "eps_clad > eps_sub: cladding orders would not all propagate in the substrate");
    cudaSetDevice(c->device);
    long long n = (long long)h * c->nx;
    const bool on_dev = is_device_ptr(eps_slab);
    // a device array is read in order on the caller's stream (after the work
    // that produced it); host arrays go through the context's own stream
    cudaStream_t s = on_dev ? (cudaStream_t)stream : c->cap_stream;
    std::vector<double> tmp;
    const double *hv = eps_slab;
    if (on_dev) {
        tmp.resize(n);
        cudaError_t e = cudaMemcpyAsync(tmp.data(), eps_slab, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return check_cuda(c, e, "read eps");
        hv = tmp.data();
    }
    for (long long i = 0; i < n; ++i)
        if (!isfinite(hv[i])) return set_err(c, APF_EINVAL, "eps_slab[%lld] is not finite", i);
    if (c->h != h || !c->d_eps) {
        if (c->d_eps) cudaFree(c->d_eps);
        c->d_eps = nullptr;
        cudaError_t e = cudaMalloc(&c->d_eps, sizeof(double) * n);
        if (e != cudaSuccess) return check_cuda(c, e, "cudaMalloc eps");
    }
    {
        cudaError_t e = cudaMemcpyAsync(c->d_eps, eps_slab, sizeof(double) * n,
                                        on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return check_cuda(c, e, on_dev ? "copy eps" : "upload eps");
    }
    bool changed = (c->h != h) || (c->eps_sub != eps_sub) || (c->eps_clad != eps_clad);
    if (changed || c->j0 != j0) graphs_reset(c);
    c->h = h; c->j0 = j0; c->eps_sub = eps_sub; c->eps_clad = eps_clad;
    c->eps_set = true;
    if (changed) c->ch_set = false;
    if (c->ch_set) return ensure_workspace(c);
    return APF_OK;
}

int apf_set_channels(apf_ctx *c, const int *m_in, int n_in, const int *m_out, int n_out) {
    if (!c) return APF_EINVAL;
    if (!c->grid_set || !c->eps_set) return set_err(c, APF_ESTATE, "apf_set_channels needs grid and eps first");
    std::vector<int> vin, vout, all;
    for (int m = -(c->nx / 2); m < c->nx - c->nx / 2; ++m) {
        double q = disp_q(c, m, c->eps_clad);
        if (q > 0.0 && q < 1.0) all.push_back(m);
    }
    if (m_in && n_in > 0) vin.assign(m_in, m_in + n_in); else vin = all;
    if (m_out && n_out > 0) vout.assign(m_out, m_out + n_out); else vout = all;
    if (vin.empty() || vout.empty()) return set_err(c, APF_EINVAL, "no channels");
    for (int m : vin) {
        double q = disp_q(c, m, c->eps_sub);
        if (!(q > 0.0 && q < 1.0)) return set_err(c, APF_EINVAL, "input order %d does not propagate in the substrate", m);
    }
    for (size_t i = 0; i < vout.size(); ++i) {
        double q = disp_q(c, vout[i], c->eps_clad);
        if (!(q > 0.0 && q < 1.0)) return set_err(c, APF_EINVAL, "output order %d does not propagate in the cladding", vout[i]);
        if (i > 0 && vout[i] <= vout[i - 1]) return set_err(c, APF_EINVAL, "output orders must be strictly ascending");
    }
    c->m_in = vin;
    c->m_out = vout;
    c->nin = (int)vin.size();
    c->nout = (int)vout.size();
    c->ch_set = true;
    graphs_reset(c);
    cudaSetDevice(c->device);
    int rc = ensure_workspace(c);
    if (rc != APF_OK) { c->ch_set = false; return rc; }
    // the orders may have changed with the same counts
    cudaMemcpyAsync(c->d_min, c->m_in.data(), sizeof(int) * c->m_in.size(), cudaMemcpyHostToDevice, c->cap_stream);
    cudaMemcpyAsync(c->d_mout, c->m_out.data(), sizeof(int) * c->m_out.size(), cudaMemcpyHostToDevice, c->cap_stream);
    cudaStreamSynchronize(c->cap_stream);
    return APF_OK;
}

int apf_get_channels(const apf_ctx *c, int *n_in, int *n_out, int *m_in, int *m_out) {
    if (!c) return APF_EINVAL;
    if (!c->ch_set) return APF_ESTATE;
    if (n_in) *n_in = c->nin;
    if (n_out) *n_out = c->nout;
    if (m_in) std::copy(c->m_in.begin(), c->m_in.end(), m_in);
    if (m_out) std::copy(c->m_out.begin(), c->m_out.end(), m_out);
    return APF_OK;
}

int apf_set_refinement(apf_ctx *c, double tol, int max_iters) {
    if (!c) return APF_EINVAL;
    if (!(tol > 0.0) || max_iters < 0 || max_iters > 100)
        return set_err(c, APF_EINVAL, "refinement: tol > 0 and 0 <= max_iters <= 100");
    c->ir_tol = tol;
    c->ir_max = max_iters;
    return APF_OK;
}

int apf_set_krylov(apf_ctx *c, int m) {
    if (!c) return APF_EINVAL;
    if (m < 0 || m > 8) return set_err(c, APF_EINVAL, "Krylov dimension %d must be in [0, 8]", m);
    if (c->precision == APF_FP64) return set_err(c, APF_EINVAL, "GMRES refinement applies to the mixed mode only");
    if (m == c->krylov_m) return APF_OK;
    c->krylov_m = m;
    if (c->ws_nx < 0) return APF_OK;  // allocated with the workspace at apf_set_channels
    cudaSetDevice(c->device);
    free_workspace(c);
    return ensure_workspace(c);
}

int apf_set_schur_storage(apf_ctx *c, int segment_rows) {
    if (!c) return APF_EINVAL;
    if (segment_rows < 0 || segment_rows > 4096)
        return set_err(c, APF_EINVAL, "segment_rows=%d must be in [0, 4096]", segment_rows);
    if (c->precision == APF_FP64 && segment_rows != 0)
        return set_err(c, APF_EINVAL, "recomputation of the slab inverses applies to the mixed mode only");
    if (segment_rows == c->schur_seg) return APF_OK;
    c->schur_seg = segment_rows;
    if (c->ws_nx < 0) return APF_OK;  // allocated with the workspace at apf_set_channels
    cudaSetDevice(c->device);
    free_workspace(c);
    return ensure_workspace(c);
}

int apf_set_elimination(apf_ctx *c, int planes, int butterfly) {
    if (!c) return APF_EINVAL;
    if (planes != 2 && planes != 3) return set_err(c, APF_EINVAL, "planes=%d must be 2 or 3", planes);
    if (butterfly != 0 && butterfly != 1) return set_err(c, APF_EINVAL, "butterfly must be 0 or 1");
    if (c->precision == APF_FP64 && (planes != 2 || butterfly))
        return set_err(c, APF_EINVAL, "split planes and the butterfly transform apply to the mixed mode only");
    if (planes == c->elim_planes && butterfly == c->butterfly) return APF_OK;
    c->elim_planes = planes;
    c->butterfly = butterfly;
    if (c->ws_nx < 0) return APF_OK;  // allocated with the workspace at apf_set_channels
    cudaSetDevice(c->device);
    free_workspace(c);
    return ensure_workspace(c);
}

int apf_set_profiling(apf_ctx *c, int enable) {
    if (!c) return APF_EINVAL;
    cudaSetDevice(c->device);
    c->prof = apf_profile{};
    if ((enable != 0) != c->prof_on) graphs_reset(c);
    c->prof_on = enable != 0;
    if (c->prof_on && c->prof_ev.empty()) {
        const int pairs = 16384;
        c->prof_ev.resize(2 * pairs);
        for (auto &e : c->prof_ev) {
            if (cudaEventCreate(&e) != cudaSuccess) return check_cuda(c, cudaGetLastError(), "profiling events");
        }
        c->prof_alg.assign(pairs, 0.0);
        c->prof_hw.assign(pairs, 0.0);
    }
    return APF_OK;
}

int apf_get_profile(const apf_ctx *c, apf_profile *p) {
    if (!c || !p) return APF_EINVAL;
    *p = c->prof;
    return APF_OK;
}

int apf_get_stats(const apf_ctx *c, apf_stats *st) {
    if (!c || !st) return APF_EINVAL;
    *st = c->stats;
    st->workspace_bytes = c->ws_bytes;
    return APF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve pipeline
// ---------------------------------------------------------------------------
void fields64(apf_ctx *c, cudaStream_t s) {
    int nf = c->cf, ncol = c->cf + c->ca;
    long long nx = c->nx, L = (long long)ncol * nx, nn = nx * nx;
    double2 *E = c->d_Ew;
    const double2 one = cmk(1, 0), zero = cmk(0, 0);
    // forward chain Y_j = G_{j-1} Y_{j-1} (forward columns; Y_0 = R_0)
    for (int j = 1; j < c->h; ++j)
        zgemm(c, false, false, nf, c->nx, c->nx, one, E + (j - 1) * L, nx, 0, c->d_G + (j - 1) * nn, nx, 0,
              zero, E + j * L, nx, 0, 1, s);
    // back substitution E_{h-1} = G_{h-1} Y_{h-1}; E_j = G_j (Y_j + E_{j+1})
    for (int j = c->h - 1; j >= 0; --j) {
        if (j == c->h - 1) launch_copy(c, c->d_T, E + j * L, L, s);
        else launch_add(c, c->d_T, E + j * L, E + (j + 1) * L, L, s);
        zgemm(c, false, false, ncol, c->nx, c->nx, one, c->d_T, nx, 0, c->d_G + j * nn, nx, 0, zero,
              E + j * L, nx, 0, 1, s);
    }
}

// Everything up to the first host synchronization: boundary elimination, slab
// elimination and the first field sweep of the current column layout (0 or 1).
// Captured once per layout into a CUDA graph.
static int main_body(apf_ctx *c, cudaStream_t s) {
    long long L = (long long)(c->cf + c->ca) * c->nx;
    cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), s);
    record_event(c, c->ev[0], s);
    launch_boundary(c, s);
    record_event(c, c->ev[1], s);
    int rc = APF_OK;
    if (c->precision == APF_FP64) {
        long long nx = c->nx, nn = nx * nx;
        for (int j = 0; j < c->h; ++j) {
            double2 *X = c->d_G + j * nn;
            launch_assemble64(c, j, X, j > 0 ? c->d_G + (j - 1) * nn : nullptr, s);
            invert_sym64(c, X, c->nx, nx, c->d_scr1, c->d_scr2, s);
        }
    } else {
        rc = mixed_eliminate(c, s);
        if (rc != APF_OK) return rc;
    }
    record_event(c, c->ev[2], s);
    launch_zero(c, c->d_Ew, sizeof(double2) * c->h * L, s);
    launch_build_rhs(c, c->d_Ew, s);
    if (c->precision == APF_FP64) fields64(c, s);
    else rc = mixed_fields_begin(c, s);
    return rc;
}

// Second pass of the conventional adjoint method (layout 2): the adjoint
// sources C_a^adj = sum_b Gamma_ba C_b on the last slab row, then the field
// sweep through the stored elimination.
static int adjoint_body(apf_ctx *c, cudaStream_t s) {
    long long L = (long long)(c->cf + c->ca) * c->nx;
    launch_zero(c, c->d_Ew, sizeof(double2) * c->h * L, s);
    launch_adjoint_rhs(c, c->d_Gam, c->d_Ew + (long long)(c->h - 1) * L, s);
    if (c->precision == APF_FP64) {
        fields64(c, s);
        return APF_OK;
    }
    return mixed_fields_begin(c, s);
}

static void set_layout(apf_ctx *c, int lay) {
    c->lay = lay;
    if (lay == 0) { c->cf = c->nin; c->ca = c->nout; c->d_Ew = c->d_E; }
    else if (lay == 1) { c->cf = c->nin; c->ca = 0; c->d_Ew = c->d_E; }
    else { c->cf = 0; c->ca = c->nin; c->d_Ew = c->d_E + (long long)c->h * c->nin * c->nx; }
}

// One pass of the solve in column layout `lay` (0: the single elimination,
// 1: the forward pass of the conventional adjoint method): elimination and
// field sweep, refinement (mixed), S readout.
static int run_solve(apf_ctx *c, cudaStream_t s, int lay = 0) {
    if (!c->grid_set || !c->eps_set || !c->ch_set)
        return set_err(c, APF_ESTATE, "solve needs apf_set_grid, apf_set_eps and apf_set_channels");
    cudaSetDevice(c->device);
    c->launches = 0;
    c->prof_used = c->prof_static;
    c->stats.refine_iters = 0;
    c->stats.residual = 0.0;
    c->fields_lay = -1;
    set_layout(c, lay);
    int rc = run_graph(c, c->g_main[lay], s, main_body);
    if (rc != APF_OK) return rc;
    if (c->precision != APF_FP64) {
        rc = mixed_refine(c, s);
        if (rc != APF_OK && rc != APF_ENOCONV) return rc;
    }
    cudaEventRecord(c->ev[3], s);
    launch_readout(c, s);
    cudaEventRecord(c->ev[4], s);
    c->fields_lay = lay;
    return rc;
}

void record_event(apf_ctx *c, cudaEvent_t e, cudaStream_t s) {
    if (c->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
}

void graphs_reset(apf_ctx *c) {
    for (int l = 0; l < 3; ++l) {
        for (GraphSlot *g : {&c->g_main[l], &c->g_resid[l], &c->g_correct[l]}) {
            if (g->exec) cudaGraphExecDestroy(g->exec);
            *g = GraphSlot{};
        }
    }
    c->prof_static = 0;
    c->prof_used = 0;
}

// Run `body` on stream s: the first time it is captured (on the context's
// capture stream) into a graph, afterwards the graph is replayed.  If
// capture is not possible the body runs eagerly.
int run_graph(apf_ctx *c, GraphSlot &g, cudaStream_t s, int (*body)(apf_ctx *, cudaStream_t)) {
    if (!c->use_graphs) return body(c, s);
    if (!g.exec) {
        long long l0 = c->launches;
        int p0 = c->prof_used;
        if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->use_graphs = false;
            return body(c, s);
        }
        c->capturing = true;
        int rc = body(c, c->cap_stream);
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (rc != APF_OK) {
            if (graph) cudaGraphDestroy(graph);
            c->launches = l0;
            c->prof_used = p0;
            return rc;
        }
        if (e != cudaSuccess || !graph || cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            g.exec = nullptr;
            c->use_graphs = false;
            c->launches = l0;
            c->prof_used = p0;
            return body(c, s);
        }
        cudaGraphDestroy(graph);
        g.launches = c->launches - l0;
        c->launches = l0;
        g.prof_lo = p0;
        g.prof_hi = c->prof_used;
        c->prof_static = c->prof_used;
    }
    cudaError_t e = cudaGraphLaunch(g.exec, s);
    if (e != cudaSuccess) return check_cuda(c, e, "graph launch");
    c->launches += g.launches;
    return APF_OK;
}

void prof_collect_range(apf_ctx *c, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) == cudaSuccess) {
            c->prof.gemm_launches++;
            c->prof.gemm_ms += ms;
            c->prof.gemm_alg_flops += c->prof_alg[i];
            c->prof.gemm_hw_flops += c->prof_hw[i];
        }
    }
    cudaGetLastError();
}

// Fold the GEMM events of launches made outside graphs into the totals.
void prof_collect(apf_ctx *c) {
    prof_collect_range(c, c->prof_static, c->prof_used);
    c->prof_used = c->prof_static;
}

static int finish(apf_ctx *c, cudaStream_t s, int rc_solve) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(c, e, "solve");
    if (c->prof_on) prof_collect(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(c, e, "kernel launch");
    int fl2[2] = {0, 0};
    cudaMemcpyAsync(fl2, c->d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int flags = fl2[0];
    c->stats.leaf_fallbacks = fl2[1];
    float ms[6] = {0};
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]);
    c->stats.ms_boundary = ms[0];
    c->stats.ms_eliminate = ms[1];
    c->stats.ms_fields = ms[2];
    c->stats.ms_readout = ms[3];
    c->stats.ms_gradient = ms[4];
    float tot = 0;
    cudaEventElapsedTime(&tot, c->ev[0], c->ev[5]);
    c->stats.ms_total = tot;
    c->stats.kernel_launches = c->launches;
    if (flags & FLAG_SINGULAR) return set_err(c, APF_ESINGULAR, "zero pivot in a diagonal-block inversion");
    if (flags & FLAG_TIMEOUT) return set_err(c, APF_ETIMEOUT, "a bounded device wait gave up");
    if (flags & FLAG_NONFINITE) return set_err(c, APF_ECUDA, "non-finite value in the elimination");
    if (rc_solve == APF_ENOCONV)
        return set_err(c, APF_ENOCONV, "refinement stopped at residual %.3e > tol %.3e", c->stats.residual, c->ir_tol);
    return APF_OK;
}

extern "C" {

int apf_solve_S(apf_ctx *c, double *S, void *stream) {
    if (!c) return APF_EINVAL;
    SolveGate gate(c->device);
    if (!S) return set_err(c, APF_EINVAL, "S is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = run_solve(c, s);
    if (rc != APF_OK && rc != APF_ENOCONV) { cudaStreamSynchronize(s); return rc; }
    cudaEventRecord(c->ev[5], s);
    size_t bytes = sizeof(double2) * (size_t)c->nin * c->nout;
    cudaMemcpyAsync(S, c->d_S, bytes, cudaMemcpyDefault, s);
    return finish(c, s, rc);
}

int apf_solve_S_grad(apf_ctx *c, int objective, const double *params, int n_params, double *S, double *f,
                     double *grad_eps, void *stream) {
    if (!c) return APF_EINVAL;
    SolveGate gate(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!grad_eps) return set_err(c, APF_EINVAL, "grad_eps is NULL");
    if (!c->grid_set || !c->eps_set || !c->ch_set)
        return set_err(c, APF_ESTATE, "solve needs apf_set_grid, apf_set_eps and apf_set_channels");
    // validate objective params before any launch
    if (objective != APF_OBJ_POWER && objective != APF_OBJ_SPLITTER)
        return set_err(c, APF_EINVAL, "unknown objective id %d", objective);
    if (!params || n_params < 2 || (int)params[1] < 1 || (int)params[1] > 16 || n_params != 2 + (int)params[1])
        return set_err(c, APF_EINVAL, "objective params must be {t, nD, d_1..d_nD} with 1 <= nD <= 16");
    int rc = run_solve(c, s);
    if (rc != APF_OK && rc != APF_ENOCONV) { cudaStreamSynchronize(s); return rc; }
    int rc2 = launch_objective(c, objective, params, n_params, s);
    if (rc2 != APF_OK) { cudaStreamSynchronize(s); return rc2; }
    rc2 = launch_gradient(c, c->d_Gam, s);
    if (rc2 != APF_OK) { cudaStreamSynchronize(s); return rc2; }
    cudaEventRecord(c->ev[5], s);
    size_t sb = sizeof(double2) * (size_t)c->nin * c->nout;
    if (S) cudaMemcpyAsync(S, c->d_S, sb, cudaMemcpyDefault, s);
    cudaMemcpyAsync(grad_eps, c->d_grad, sizeof(double) * c->h * c->nx, cudaMemcpyDefault, s);
    double fh = 0.0;
    cudaMemcpyAsync(&fh, c->d_f, sizeof(double), cudaMemcpyDeviceToHost, s);
    int r = finish(c, s, rc);
    if (f) *f = fh;
    return r;
}

// The conventional adjoint method (paper Supplement Sec. 1, Eq. S1) on the same
// elimination: forward fields of the n_in inputs (with their own refinement),
// S, f and Gamma, then a second sweep of n_in adjoint fields whose sources
// C_a^adj = sum_b Gamma_ba C_b are known only after Gamma, and the elementwise
// contraction of forward and adjoint fields.
static int adjoint_method(apf_ctx *c, int objective, const double *params, int n_params, cudaStream_t s,
                          int *rc_solve) {
    int rc = run_solve(c, s, 1);
    if (rc != APF_OK && rc != APF_ENOCONV) return rc;
    *rc_solve = rc;
    const int it1 = c->stats.refine_iters;
    const double res1 = c->stats.residual;
    rc = launch_objective(c, objective, params, n_params, s);
    if (rc != APF_OK) return rc;
    c->fields_lay = -1;
    set_layout(c, 2);
    rc = run_graph(c, c->g_main[2], s, adjoint_body);
    if (rc != APF_OK) return rc;
    if (c->precision != APF_FP64) {
        rc = mixed_refine(c, s);
        if (rc != APF_OK && rc != APF_ENOCONV) return rc;
        if (rc == APF_ENOCONV) *rc_solve = rc;
    }
    c->stats.refine_iters += it1;
    c->stats.residual = std::max(c->stats.residual, res1);
    launch_gradient_adjoint(c, c->d_E, c->d_Ew, s);
    set_layout(c, 1);
    c->fields_lay = 1;
    return APF_OK;
}

int apf_solve_S_grad_adjoint(apf_ctx *c, int objective, const double *params, int n_params, double *S, double *f,
                             double *grad_eps, void *stream) {
    if (!c) return APF_EINVAL;
    SolveGate gate(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!grad_eps) return set_err(c, APF_EINVAL, "grad_eps is NULL");
    if (!c->grid_set || !c->eps_set || !c->ch_set)
        return set_err(c, APF_ESTATE, "solve needs apf_set_grid, apf_set_eps and apf_set_channels");
    if (objective != APF_OBJ_POWER && objective != APF_OBJ_SPLITTER)
        return set_err(c, APF_EINVAL, "unknown objective id %d", objective);
    if (!params || n_params < 2 || (int)params[1] < 1 || (int)params[1] > 16 || n_params != 2 + (int)params[1])
        return set_err(c, APF_EINVAL, "objective params must be {t, nD, d_1..d_nD} with 1 <= nD <= 16");
    int rc_solve = APF_OK;
    int rc = adjoint_method(c, objective, params, n_params, s, &rc_solve);
    if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    cudaEventRecord(c->ev[5], s);
    size_t sb = sizeof(double2) * (size_t)c->nin * c->nout;
    if (S) cudaMemcpyAsync(S, c->d_S, sb, cudaMemcpyDefault, s);
    cudaMemcpyAsync(grad_eps, c->d_grad, sizeof(double) * c->h * c->nx, cudaMemcpyDefault, s);
    double fh = 0.0;
    cudaMemcpyAsync(&fh, c->d_f, sizeof(double), cudaMemcpyDeviceToHost, s);
    int r = finish(c, s, rc_solve);
    if (f) *f = fh;
    return r;
}

// Several designs in one call: the mixed pipeline with every launch of the
// elimination, the field sweeps and the gradient shared by the designs.
static bool same_problem(const apf_ctx *a, const apf_ctx *b) {
    return a->device == b->device && a->precision == b->precision && a->nx == b->nx && a->ny == b->ny &&
           a->npml_bot == b->npml_bot && a->npml_top == b->npml_top && a->lambda_px == b->lambda_px &&
           a->R0 == b->R0 && a->power == b->power && a->h == b->h && a->j0 == b->j0 && a->eps_sub == b->eps_sub &&
           a->eps_clad == b->eps_clad && a->m_in == b->m_in && a->m_out == b->m_out && a->ir_tol == b->ir_tol &&
           a->ir_max == b->ir_max && a->krylov_m == b->krylov_m && a->schur_seg == b->schur_seg &&
           a->butterfly == b->butterfly && a->elim_planes == b->elim_planes;
}

int apf_solve_S_grad_batch(apf_ctx *const *ctx, int nb, int objective, const double *params, int n_params,
                           double *const *S, double *f, double *const *grad_eps, void *stream) {
    if (!ctx || nb < 1 || nb > APF_MAX_BATCH || !grad_eps)
        return set_err(nullptr, APF_EINVAL, "apf_solve_S_grad_batch: need 1..%d contexts and grad_eps", APF_MAX_BATCH);
    for (int b = 0; b < nb; ++b) {
        if (!ctx[b] || !grad_eps[b]) return set_err(nullptr, APF_EINVAL, "apf_solve_S_grad_batch: NULL entry %d", b);
        for (int a = 0; a < b; ++a)
            if (ctx[a] == ctx[b]) return set_err(ctx[b], APF_EINVAL, "a context appears twice in the batch");
    }
    SolveGate gate(ctx[0]->device);
    apf_ctx *c0 = ctx[0];
    for (int b = 0; b < nb; ++b) {
        apf_ctx *c = ctx[b];
        if (!c->grid_set || !c->eps_set || !c->ch_set || c->ws_nx < 0)
            return set_err(c, APF_ESTATE, "solve needs apf_set_grid, apf_set_eps and apf_set_channels");
        if (!same_problem(c0, c))
            return set_err(c, APF_EINVAL, "batch entry %d: grid, slab rows, channels or settings differ from entry 0", b);
    }
    if (objective != APF_OBJ_POWER && objective != APF_OBJ_SPLITTER)
        return set_err(c0, APF_EINVAL, "unknown objective id %d", objective);
    if (!params || n_params < 2 || (int)params[1] < 1 || (int)params[1] > 16 || n_params != 2 + (int)params[1])
        return set_err(c0, APF_EINVAL, "objective params must be {t, nD, d_1..d_nD} with 1 <= nD <= 16");
    cudaStream_t s = (cudaStream_t)stream;
    if (c0->precision == APF_FP64 || c0->krylov_m > 0) {
        // float64 (SIMT products, already grid-filling) and GMRES refinement: one design at a time
        for (int b = 0; b < nb; ++b) {
            int rc = apf_solve_S_grad(ctx[b], objective, params, n_params, S ? S[b] : nullptr, f ? f + b : nullptr,
                                      grad_eps[b], stream);
            if (rc != APF_OK) return rc;
        }
        return APF_OK;
    }
    for (int b = 1; b < nb; ++b)
        if (!mixed_batch_compatible(c0, ctx[b]))
            return set_err(ctx[b], APF_EINVAL, "batch entry %d: mixed-mode workspace settings differ", b);
    cudaSetDevice(c0->device);
    for (int b = 0; b < nb; ++b) {
        apf_ctx *c = ctx[b];
        c->launches = 0;
        c->prof_used = c->prof_static;
        c->stats.refine_iters = 0;
        c->stats.residual = 0.0;
        c->fields_lay = -1;
        set_layout(c, 0);
        cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), s);
    }
    cudaEventRecord(c0->ev[0], s);
    for (int b = 0; b < nb; ++b) launch_boundary(ctx[b], s);
    cudaEventRecord(c0->ev[1], s);
    int rc = mixed_eliminate_n(ctx, nb, s);
    if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    cudaEventRecord(c0->ev[2], s);
    for (int b = 0; b < nb; ++b) {
        apf_ctx *c = ctx[b];
        launch_zero(c, c->d_Ew, sizeof(double2) * c->h * (long long)(c->cf + c->ca) * c->nx, s);
        launch_build_rhs(c, c->d_Ew, s);
    }
    rc = mixed_fields_begin_n(ctx, nb, s);
    if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    int rcs[APF_MAX_BATCH] = {};
    rc = mixed_refine_n(ctx, nb, s, rcs);
    if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    cudaEventRecord(c0->ev[3], s);
    for (int b = 0; b < nb; ++b) {
        launch_readout(ctx[b], s);
        rc = launch_objective(ctx[b], objective, params, n_params, s);
        if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    }
    cudaEventRecord(c0->ev[4], s);
    rc = mixed_gradient_n(ctx, nb, s);
    if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    cudaEventRecord(c0->ev[5], s);
    std::vector<double> fh(nb, 0.0);
    std::vector<int> fl(2 * nb, 0);
    for (int b = 0; b < nb; ++b) {
        apf_ctx *c = ctx[b];
        const size_t sb = sizeof(double2) * (size_t)c->nin * c->nout;
        if (S && S[b]) cudaMemcpyAsync(S[b], c->d_S, sb, cudaMemcpyDefault, s);
        cudaMemcpyAsync(grad_eps[b], c->d_grad, sizeof(double) * c->h * c->nx, cudaMemcpyDefault, s);
        cudaMemcpyAsync(&fh[b], c->d_f, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&fl[2 * b], c->d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(c0, e, "batched solve");
    if (c0->prof_on) prof_collect(c0);
    float ms[6] = {0};
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&ms[i], c0->ev[i], c0->ev[i + 1]);
    float tot = 0;
    cudaEventElapsedTime(&tot, c0->ev[0], c0->ev[5]);
    int ret = APF_OK;
    for (int b = 0; b < nb; ++b) {
        apf_ctx *c = ctx[b];
        c->stats.ms_boundary = ms[0];
        c->stats.ms_eliminate = ms[1];
        c->stats.ms_fields = ms[2];
        c->stats.ms_readout = ms[3];
        c->stats.ms_gradient = ms[4];
        c->stats.ms_total = tot;
        c->stats.kernel_launches = c->launches;
        c->stats.leaf_fallbacks = fl[2 * b + 1];
        c->fields_lay = 0;
        if (f) f[b] = fh[b];
        int r = APF_OK;
        if (fl[2 * b] & FLAG_SINGULAR) r = set_err(c, APF_ESINGULAR, "zero pivot in a diagonal-block inversion");
        else if (fl[2 * b] & FLAG_TIMEOUT) r = set_err(c, APF_ETIMEOUT, "a bounded device wait gave up");
        else if (fl[2 * b] & FLAG_NONFINITE) r = set_err(c, APF_ECUDA, "non-finite value in the elimination");
        else if (rcs[b] == APF_ENOCONV)
            r = set_err(c, APF_ENOCONV, "refinement stopped at residual %.3e > tol %.3e", c->stats.residual, c->ir_tol);
        if (r != APF_OK && (ret == APF_OK || ret == APF_ENOCONV)) ret = r;
    }
    return ret;
}

int apf_grad_from_gamma(apf_ctx *c, const double *Gamma, double *grad_eps, void *stream) {
    if (!c) return APF_EINVAL;
    SolveGate gate(c->device);
    if (!Gamma || !grad_eps) return set_err(c, APF_EINVAL, "Gamma / grad_eps is NULL");
    if (!c->ch_set || c->ws_nx < 0) return set_err(c, APF_ESTATE, "apf_grad_from_gamma needs a previous solve");
    if (c->fields_lay != 0)
        return set_err(c, APF_ESTATE, "apf_grad_from_gamma needs the fields of apf_solve_S or apf_solve_S_grad");
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(c->device);
    size_t sb = sizeof(double2) * (size_t)c->nin * c->nout;
    cudaMemcpyAsync(c->d_Gam, Gamma, sb, cudaMemcpyDefault, s);
    c->launches = 0;
    cudaEventRecord(c->ev[4], s);
    int rc = launch_gradient(c, c->d_Gam, s);
    if (rc != APF_OK) { cudaStreamSynchronize(s); return rc; }
    cudaEventRecord(c->ev[5], s);
    cudaMemcpyAsync(grad_eps, c->d_grad, sizeof(double) * c->h * c->nx, cudaMemcpyDefault, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return check_cuda(c, e, "grad_from_gamma");
    if (c->prof_on) prof_collect(c);
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]);
    c->stats.ms_gradient = ms;
    return APF_OK;
}


int apf_substrate_orders(const apf_ctx *c, int *n, int *m) {
    if (!c) return APF_EINVAL;
    if (!c->grid_set || !c->eps_set) return APF_ESTATE;
    int cnt = 0;
    for (int o = -(c->nx / 2); o < c->nx - c->nx / 2; ++o) {
        double q = disp_q(c, o, c->eps_sub);
        if (q > 0.0 && q < 1.0) {
            if (m) m[cnt] = o;
            ++cnt;
        }
    }
    if (n) *n = cnt;
    return APF_OK;
}

int apf_reflection(apf_ctx *c, const int *m_ref, int n_ref, double *R, void *stream) {
    if (!c) return APF_EINVAL;
    if (!R) return set_err(c, APF_EINVAL, "R is NULL");
    if (!c->ch_set || c->ws_nx < 0 || c->fields_lay < 0)
        return set_err(c, APF_ESTATE, "apf_reflection needs a previous solve");
    std::vector<int> ord;
    if (m_ref && n_ref > 0) {
        if (n_ref > c->nx) return set_err(c, APF_EINVAL, "n_ref=%d exceeds nx=%d", n_ref, c->nx);
        ord.assign(m_ref, m_ref + n_ref);
        for (int o : ord) {
            double q = disp_q(c, o, c->eps_sub);
            if (!(q > 0.0 && q < 1.0))
                return set_err(c, APF_EINVAL, "reflection order %d does not propagate in the substrate", o);
        }
    } else {
        for (int o = -(c->nx / 2); o < c->nx - c->nx / 2; ++o) {
            double q = disp_q(c, o, c->eps_sub);
            if (q > 0.0 && q < 1.0) ord.push_back(o);
        }
    }
    const int nr = (int)ord.size();
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(c->d_mref, ord.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return check_cuda(c, e, "upload reflection orders");
    launch_source_row(c, c->d_qsrc, s);
    // first slab row of the forward columns, to the Fourier basis
    launch_fft(c, c->d_E, c->d_fft, c->nx, c->nin, c->nx, c->nx, -1, 1.0 / sqrt((double)c->nx), s);
    launch_reflection(c, c->d_fft, c->d_qsrc, c->d_mref, nr, c->d_refl, s);
    e = cudaMemcpyAsync(R, c->d_refl, sizeof(double2) * (size_t)nr * c->nin, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(c, e, "reflection");
    return APF_OK;
}

int apf_reverse_S(apf_ctx *c, double *S_rev, void *stream) {
    if (!c) return APF_EINVAL;
    if (!S_rev) return set_err(c, APF_EINVAL, "S_rev is NULL");
    if (!c->ch_set || c->ws_nx < 0 || c->fields_lay != 0)
        return set_err(c, APF_ESTATE, "apf_reverse_S needs the fields of apf_solve_S or apf_solve_S_grad");
    std::vector<int> rmap(c->nout);
    for (int q = 0; q < c->nout; ++q) {
        int hit = -1;
        for (int b = 0; b < c->nout; ++b)
            if (c->m_out[b] == -c->m_out[q]) { hit = b; break; }
        if (hit < 0)
            return set_err(c, APF_EINVAL, "reverse transmission needs order %d in the output set (output %d)",
                           -c->m_out[q], c->m_out[q]);
        rmap[q] = hit;
    }
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int ncol = c->nin + c->nout;
    cudaError_t e = cudaMemcpyAsync(c->d_rmap, rmap.data(), sizeof(int) * c->nout, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return check_cuda(c, e, "upload order map");
    launch_fft(c, c->d_E, c->d_fft, c->nx, ncol, c->nx, c->nx, -1, 1.0 / sqrt((double)c->nx), s);
    launch_reverse_S(c, c->d_fft, c->d_rmap, c->d_srev, s);
    e = cudaMemcpyAsync(S_rev, c->d_srev, sizeof(double2) * (size_t)c->nin * c->nout, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(c, e, "reverse S");
    return APF_OK;
}

}  // extern "C"
