// Internal declarations shared by the CUDA translation units of libapf.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/apf.h"

// ---------------------------------------------------------------------------
// complex float64 helpers (interleaved double2)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm (avoids overflow for large |b|).
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ double2 cinv(double2 b) { return cdiv(make_double2(1.0, 0.0), b); }

// complex float32 helpers
__host__ __device__ __forceinline__ float2 fmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------------------
// Grid description passed by value to kernels.
// ---------------------------------------------------------------------------
struct GridDev {
    int nx, ny, npml_bot, npml_top;
    int j0, h, jsrc, jout;
    double k;            // 2 pi / lambda_px
    double eps_sub, eps_clad;
    double R0, power;
};

// Error flag bits written by kernels into ctx->d_flags[0].
enum { FLAG_SINGULAR = 1, FLAG_NONFINITE = 2, FLAG_TIMEOUT = 4 };

// Sizes of the mixed-mode (tensor-core) workspace; defined in mixed.cu.
struct MixedWork;

// A captured CUDA graph for one phase of the solve.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;  // kernels per replay
    int prof_lo = 0, prof_hi = 0;  // profiling event pairs owned by this graph
};

struct apf_ctx {
    int device = 0;
    int precision = APF_FP64;
    // grid
    bool grid_set = false;
    int nx = 0, ny = 0, npml_bot = 0, npml_top = 0;
    double lambda_px = 0, k = 0, R0 = 1e-8, power = 3.0;
    // slab
    bool eps_set = false;
    int h = 0, j0 = 0;
    double eps_sub = 1, eps_clad = 1;
    // channels
    bool ch_set = false;
    std::vector<int> m_in, m_out;
    int nin = 0, nout = 0;  // channel counts used by all device-side code
    // refinement
    double ir_tol = 1e-10;
    int ir_max = 40;
    int krylov_m = 0;  // mixed mode: GMRES(m) refinement when > 0
    int schur_seg = 0; // mixed mode: recompute the slab inverses in segments of this many rows (0: store all)
    int butterfly = 0; // mixed mode: symmetric random butterfly transform of every slab block before inversion
    int elim_planes = 2; // mixed mode: bf16 split planes of the elimination and sweep products (2: bf16x3, 3: bf16x6)
    // workspace signature
    int ws_nx = -1, ws_ny = -1, ws_h = -1, ws_min = -1, ws_mout = -1;
    long long ws_bytes = 0;
    std::vector<void *> allocs;
    // device buffers (float64 path, also used by the mixed path)
    double *d_eps = nullptr;     // h*nx
    int *d_min = nullptr, *d_mout = nullptr;
    double2 *d_modes = nullptr;  // 4*nx: sigma_bot, sigma_top, fac_bot, tau
    double2 *d_stretch = nullptr; // 2*(ny+1): s_j and 1/s_{j-1/2}
    double2 *d_coef = nullptr;   // n_in + n_out: beta_a, w_b
    double2 *d_circ = nullptr;   // 2*nx: circulant generators of Sigma_bot, Sigma_top
    double2 *d_tw = nullptr;     // nx/2 twiddles exp(-2 pi i k / nx)
    double2 *d_G = nullptr;      // h*nx*nx   (float64 mode)
    double2 *d_scr1 = nullptr, *d_scr2 = nullptr;  // recursion scratch, nx*nx/2 each
    double2 *d_E = nullptr;      // h*ncol*nx fields, [row][column][x]
    double2 *d_T = nullptr;      // ncol*nx temp
    double2 *d_R = nullptr;      // h*ncol*nx residual (mixed)
    double2 *d_S = nullptr, *d_Gam = nullptr;  // n_out*n_in
    double2 *d_qsrc = nullptr;   // nx: source-row coefficient q[m] of the substrate side
    double2 *d_refl = nullptr;   // nx*n_in: reflection block (apf_reflection)
    double2 *d_srev = nullptr;   // n_in*n_out: transmission from the cladding side (apf_reverse_S)
    int *d_mref = nullptr;       // nx: reflection orders
    int *d_rmap = nullptr;       // n_out: adjoint column of the opposite output order
    double2 *d_Q = nullptr;      // h*n_out*nx
    double2 *d_fft = nullptr;    // ncol*nx
    double *d_grad = nullptr;    // h*nx
    double *d_f = nullptr;       // scalars: f, residual norms
    double *d_colnorm = nullptr; // 2*ncol: ||R||, ||r|| per column
    int *d_flags = nullptr;
    int *d_pairs = nullptr;      // objective (b, a) pairs
    MixedWork *mw = nullptr;
    // ridge parametrization (apf_set_ridges): edges and the slab they define
    double *d_edges = nullptr, *d_ridge_g = nullptr;  // n_edges each
    double *d_ridge_eps = nullptr;                     // h*nx: generated eps, then host grad_eps staging
    int ridge_n = 0, ridge_cap = 0, ridge_h = 0, ridge_mirror = 0;
    long long ridge_eps_cap = 0;
    double ridge_eps_r = 0, ridge_eps_b = 0;
    // Column layout of the slab fields being swept: cf forward columns (sources
    // on the first slab row) followed by ca adjoint columns (sources on the last
    // slab row), stored at d_Ew as [row][cf + ca][x].  The single-elimination
    // solve sweeps (n_in, n_out) at d_E (layout 0).  The conventional adjoint
    // method sweeps (n_in, 0) at d_E (layout 1), then (0, n_in) at
    // d_E + h n_in nx (layout 2).
    int lay = 0, cf = 0, ca = 0;
    double2 *d_Ew = nullptr;
    int fields_lay = -1;  // layout of the fields the last solve left (0 or 1; -1: none)
    // CUDA graphs (captured on cap_stream, replayed on the caller's stream), one per layout
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = true;
    bool capturing = false;
    GraphSlot g_main[3], g_resid[3], g_correct[3];
    // GEMM launch profiling
    int prof_static = 0;  // pairs reserved by captured graphs
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;      // pairs
    std::vector<double> prof_alg, prof_hw; // per recorded pair
    int prof_used = 0;
    apf_profile prof{};
    // stats
    apf_stats stats{};
    long long launches = 0;
    cudaEvent_t ev[8] = {};
    std::string err;
};

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
#define APF_LAUNCH(ctx, kernel, grid, block, smem, stream, ...)              \
    do {                                                                      \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);           \
        (ctx)->launches++;                                                    \
    } while (0)

GridDev make_grid(const apf_ctx *c);

// boundary.cu
void launch_boundary(apf_ctx *c, cudaStream_t s);
void launch_build_rhs(apf_ctx *c, double2 *E, cudaStream_t s);
void launch_adjoint_rhs(apf_ctx *c, const double2 *Gamma, double2 *E, cudaStream_t s);
void launch_source_row(apf_ctx *c, double2 *q, cudaStream_t s);
void launch_reflection(apf_ctx *c, const double2 *fft0, const double2 *q, const int *m_ref, int n_ref, double2 *R,
                       cudaStream_t s);
void launch_reverse_S(apf_ctx *c, const double2 *fft0, const int *rmap, double2 *Srev, cudaStream_t s);
void launch_twiddles(apf_ctx *c, cudaStream_t s);
void launch_fft(apf_ctx *c, const double2 *in, double2 *out, int n, int batch, long long in_stride,
                long long out_stride, int sign, double scale, cudaStream_t s);
int fft_smem_bytes(int n);

// slab64.cu
void launch_assemble64(apf_ctx *c, int row, double2 *X, const double2 *Gprev, cudaStream_t s);
void zgemm(apf_ctx *c, bool ta, bool tb, int M, int N, int K, double2 alpha,
           const double2 *A, long long lda, long long sA,
           const double2 *B, long long ldb, long long sB, double2 beta,
           double2 *C, long long ldc, long long sC, int batch, cudaStream_t s);
void invert_sym64(apf_ctx *c, double2 *X, int n, long long ld, double2 *scr1, double2 *scr2, cudaStream_t s);
void launch_add(apf_ctx *c, double2 *T, const double2 *a, const double2 *b, long long n, cudaStream_t s);
void launch_copy(apf_ctx *c, double2 *dst, const double2 *src, long long n, cudaStream_t s);
void launch_zero(apf_ctx *c, void *dst, long long bytes, cudaStream_t s);

void fields64(apf_ctx *c, cudaStream_t s);

// readout.cu
void launch_readout(apf_ctx *c, cudaStream_t s);  // S from fields
int launch_objective(apf_ctx *c, int objective, const double *params, int n_params, cudaStream_t s);
int launch_gradient(apf_ctx *c, const double2 *Gamma, cudaStream_t s);
void launch_gradient_adjoint(apf_ctx *c, const double2 *Fw, const double2 *Lam, cudaStream_t s);
int mixed_gradient(apf_ctx *c, const double2 *Gamma, cudaStream_t s);

// mixed.cu
int mixed_alloc(apf_ctx *c);
void mixed_free(apf_ctx *c);
int mixed_eliminate(apf_ctx *c, cudaStream_t s);
int mixed_fields_begin(apf_ctx *c, cudaStream_t s);
int mixed_refine(apf_ctx *c, cudaStream_t s);
// the same steps for a batch of designs (shared launches), see apf_solve_S_grad_batch
constexpr int APF_MAX_BATCH = 16;
int mixed_eliminate_n(apf_ctx *const *cs, int nb, cudaStream_t s);
int mixed_fields_begin_n(apf_ctx *const *cs, int nb, cudaStream_t s);
int mixed_refine_n(apf_ctx *const *cs, int nb, cudaStream_t s, int *rcs);
int mixed_gradient_n(apf_ctx *const *cs, int nb, cudaStream_t s);
bool mixed_batch_compatible(const apf_ctx *a, const apf_ctx *b);

// Solve calls on one device run one at a time: a call waits in the
// constructor while another thread's call on the same device is inside
// (nested calls on one thread hold one slot).  Every such call synchronises
// its stream before returning, so the library never has two solves' kernels
// on one GPU together, whatever the number of host threads.
struct SolveGate {
    explicit SolveGate(int device);
    ~SolveGate();
    SolveGate(const SolveGate &) = delete;
    SolveGate &operator=(const SolveGate &) = delete;

  private:
    int dev_;
    bool held_;
};

int set_err(apf_ctx *c, int code, const char *fmt, ...);
void prof_collect(apf_ctx *c);
void prof_collect_range(apf_ctx *c, int lo, int hi);
void record_event(apf_ctx *c, cudaEvent_t e, cudaStream_t s);
void graphs_reset(apf_ctx *c);
int run_graph(apf_ctx *c, GraphSlot &g, cudaStream_t s, int (*body)(apf_ctx *, cudaStream_t));
void boundary_init_attrs();
int tc_init();
void slab64_init_attrs();
void mixed_init_attrs();
int check_cuda(apf_ctx *c, cudaError_t e, const char *what);
bool is_device_ptr(const void *p);

// ridges.cu
void ridges_free(apf_ctx *c);
