/*
 * apf.h -- C ABI of the GB300 augmented-partial-factorization solver.
 *
 * Problem (paper Sec. 2, first paragraph and Fig. 1a): given the relative
 * permittivity of a 2D TM structure, return the generalized scattering
 * matrix S = C A^-1 B - D over many input and output channels, and the
 * gradient of an objective f(S) with respect to the permittivity of every
 * design pixel (Eq. 1 with Eqs. 2-4: dA/dp_k is diagonal and rank one for a
 * pixel, so the whole gradient comes from C A^-1 U and U^T A^-1 B in the same
 * elimination).
 *
 * Geometry and conventions
 *   - Grid nx (periodic, x) by ny rows (y); unit pixel; vacuum wavelength
 *     lambda_px pixels, k = 2 pi / lambda_px.  Rows [0, npml_bot) and
 *     [ny - npml_top, ny) are graded PMLs: s(y) = 1 + i a (d/L)^p,
 *     a = -(p+1) ln(R0) / (2 k sqrt(eps_side) L), d measured from the
 *     half-integer interface row, Dirichlet walls beyond.
 *   - A = -d2/dx2 - d/dy (1/s) d/dy - k^2 eps, multiplied through by s and by
 *     dx^2 (complex symmetric; 5-point stencil).
 *   - Substrate (eps_sub) fills rows below the slab, cladding (eps_clad)
 *     rows above; the design slab is rows [j0, j0+h) with eps_slab[j][x].
 *   - Channels: Fourier orders u_m(x) = exp(2 pi i m x/nx)/sqrt(nx).  Input a:
 *     unit-flux source -2i sqrt(nu_a) u_{m_a} on row npml_bot; output b:
 *     projection sqrt(nu_b) u_{m_b}^H on row ny-npml_top-1; nu = sin(k_y) of
 *     the 5-point dispersion in the substrate / cladding; D = 0.
 *   - Gradient: df/deps_k = 2 Re sum_{ba} Gamma_ba dS_ba/deps_k with
 *     Gamma = df/dS the Wirtinger derivative (Eq. 1); dA/deps_k = -k^2.
 *
 * Memory
 *   - All arrays are row-major.  Complex arrays are interleaved (re, im)
 *     float64 pairs.  Array arguments may be host or device pointers (the
 *     library asks the CUDA runtime which); results land where the pointer
 *     points.  The caller owns all argument buffers; the context owns its
 *     device workspace, allocated by the apf_set_* calls (never by a solve).
 *   - A solve enqueues its kernels on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream) and synchronizes that stream before returning,
 *     so host outputs are valid on return.
 *
 * Errors
 *   - Every int-returning call returns APF_OK (0) or a negative APF_E* code;
 *     apf_last_error() gives a one-line message for the most recent failure.
 *   - Size/argument checks run on the host before any launch (APF_EINVAL).
 *   - A context is single-threaded: calls on one context must not overlap.
 *
 * Threads
 *   - Different contexts may be used from different host threads.  Calls
 *     that run solve kernels (apf_solve_S, apf_solve_S_grad,
 *     apf_solve_S_grad_adjoint, apf_solve_S_grad_batch, apf_grad_from_gamma,
 *     apf_solve_S_noalloc) run one at a time per device: a call blocks on
 *     the host while another thread's call on the same device is inside the
 *     library.  Several designs at once go through apf_solve_S_grad_batch.
 */
#ifndef APF_H
#define APF_H

#ifdef __cplusplus
extern "C" {
#endif

#define APF_OK 0
#define APF_EINVAL (-1)     /* bad argument, size, or non-finite permittivity */
#define APF_ENOMEM (-2)     /* device allocation failed */
#define APF_ESINGULAR (-3)  /* a zero pivot in a diagonal-block inversion */
#define APF_ENOCONV (-4)    /* refinement stopped above tolerance (results returned) */
#define APF_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define APF_ECUDA (-6)      /* CUDA runtime error */
#define APF_ESTATE (-7)     /* call order: grid, permittivity or channels not set */

/* Arithmetic of the slab elimination (the paper factors in float64; the mixed
   modes are this library's: low-precision products plus float64 refinement). */
#define APF_FP64 0          /* everything in float64 */
#define APF_MIXED_TF32 1    /* reserved: TF32 tensor-core products are not built;
                               apf_create returns APF_EINVAL for it */
#define APF_MIXED_BF16X3 2  /* tensor-core bf16x3 products, fp32 accumulation,
                               float64 iterative refinement of the fields */

/* Objectives for apf_solve_S_grad (relative diffraction orders d = m_out - m_in). */
#define APF_OBJ_POWER 1     /* f = sum_a sum_{d in D} |S_{a+d,a}|^2 */
#define APF_OBJ_SPLITTER 2  /* f = sum_a sum_{d in D} (|S_{a+d,a}|^2 - t)^2   (Eq. 5) */

typedef struct apf_ctx apf_ctx;

typedef struct {
    double R0;     /* normal-incidence PML round-trip reflection (default 1e-8) */
    double power;  /* grading exponent p (default 3) */
} apf_pml_params;

typedef struct {
    int refine_iters;       /* refinement sweeps taken by the last solve */
    double residual;        /* max over columns of ||r||/||R|| after the last solve */
    double ms_total;        /* device time of the last solve, milliseconds */
    double ms_boundary;     /* per-mode boundary elimination + channel set-up */
    double ms_eliminate;    /* slab block-Schur elimination (inversions) */
    double ms_fields;       /* right-hand-side sweeps (+ refinement) */
    double ms_readout;      /* S, f, Gamma */
    double ms_gradient;     /* adjoint contraction */
    long long kernel_launches; /* kernels launched by the last solve */
    long long workspace_bytes; /* device bytes held by the context */
    int leaf_fallbacks;     /* mixed mode: 128 x 128 diagonal blocks whose recursive
                               inversion failed its self-check and were redone with
                               pivoting over the whole block (last solve) */
} apf_stats;

/* Create a context on CUDA device `cuda_device` with APF_FP64 or
   APF_MIXED_BF16X3 arithmetic.  *out receives the handle (NULL on failure).
   The context stands for one instance of the paper's problem (Sec. 2, first
   paragraph: the operator A, the inputs B and the outputs C of one
   structure); it owns every device array the solves need.  APF_EINVAL for an
   unknown precision or a device index out of range, APF_ECUDA without a
   CUDA device; the mixed mode also needs an sm_103 GPU (APF_EINVAL). */
int apf_create(apf_ctx **out, int cuda_device, int precision);

/* Free the context and its device workspace.  NULL is a no-op. */
void apf_destroy(apf_ctx *ctx);

/* Grid (paper Sec. 2 operator; readings in the header comment).  nx must be
   a power of two in [8, 8192]; npml_bot, npml_top >= 1; lambda_px > 2.
   pml may be NULL for the defaults.  Invalidates permittivity and channels. */
int apf_set_grid(apf_ctx *ctx, int nx, int ny, int npml_bot, int npml_top,
                 double lambda_px, const apf_pml_params *pml);

/* Design slab and background media: the relative permittivity eps_r(r)
   that the operator A of paper Sec. 2 contains (-k^2 eps on its diagonal),
   with the design variables p_k of Eq. 1 being the slab pixels.
   eps_slab: h*nx float64, [row][x], host or device, real and finite
   (APF_EINVAL otherwise, before anything is changed).  j0 < 0 centres the
   slab between the PMLs; otherwise the source row npml_bot < j0 and
   j0+h <= ny-npml_top-1.  A device-resident eps_slab is read in order on
   `stream` (a cudaStream_t, NULL = the legacy default stream): pass the
   stream whose work produced it; the call synchronizes that stream before it
   returns, so the caller may then reuse or free eps_slab.  Host arrays are
   copied before return as well. */
int apf_set_eps(apf_ctx *ctx, const double *eps_slab, int j0, int h,
                double eps_sub, double eps_clad, void *stream);

/* Channel orders (host int arrays).  NULL (or n = 0) selects every order
   that propagates in the cladding (paper Sec. 3: all angles within the range
   of interest, spaced 2 pi / W).  Inputs must propagate in the substrate,
   outputs in the cladding.  Requires set_grid and set_eps. */
int apf_set_channels(apf_ctx *ctx, const int *m_in, int n_in,
                     const int *m_out, int n_out);

/* Query the channel counts; m_in / m_out (host, may be NULL) receive the
   orders (n_in resp. n_out ints). */
int apf_get_channels(const apf_ctx *ctx, int *n_in, int *n_out, int *m_in, int *m_out);

/* S = C A^-1 B (n_out x n_in complex128, [b][a]): the scattering matrix of
   paper Sec. 2 (first paragraph; D = 0 for transmission), all input and
   output channels from one elimination.  Keeps the slab fields so that
   apf_grad_from_gamma can follow.  APF_ESTATE before apf_set_grid,
   apf_set_eps and apf_set_channels; APF_ENOCONV (mixed mode) returns S
   from a refinement that stopped above its tolerance. */
int apf_solve_S(apf_ctx *ctx, double *S, void *stream);

/* S, f and df/deps (h*nx float64) for a built-in objective.
   params = {t, nD, d_1, ..., d_nD} (as doubles), n_params = 2 + nD.
   f is a host pointer (may be NULL); S and grad_eps may be host or device. */
int apf_solve_S_grad(apf_ctx *ctx, int objective, const double *params, int n_params,
                     double *S, double *f, double *grad_eps, void *stream);

/* The paper's conventional adjoint method (Supplement Sec. 1, Eq. S1), the
   baseline that APF is measured against (Supplement Table S1), on the same
   structured elimination: the M_in forward fields A^-1 B_a, S and Gamma =
   df/dS, then M_in adjoint fields with the sources C_a^adj = sum_b Gamma_ba
   C_b (known only after Gamma, so a second sweep), and df/deps_k =
   2 k^2 Re sum_a (A^-1 C_a^adj^T)_k (A^-1 B_a)_k.  Same arguments, results and
   errors as apf_solve_S_grad (S, f and df/deps agree with it to rounding);
   in mixed mode each of the two sweeps is refined to the tolerance of
   apf_set_refinement.  The adjoint fields it leaves are not those
   apf_grad_from_gamma and apf_reverse_S need (APF_ESTATE until the next
   apf_solve_S or apf_solve_S_grad). */
int apf_solve_S_grad_adjoint(apf_ctx *ctx, int objective, const double *params, int n_params,
                             double *S, double *f, double *grad_eps, void *stream);

/* S, f and df/deps for nb independent designs in one call (nb <= 16; the
   paper's Sec. 3 runs 1000 independent starts, and line searches try several
   designs per iteration).  ctx[0..nb) are distinct contexts, each prepared
   by apf_set_grid, apf_set_eps (its own permittivity) and apf_set_channels,
   with the same grid, slab rows, channel orders, precision and refinement /
   storage settings (APF_EINVAL otherwise).  In mixed mode every launch of the
   slab elimination, the field sweeps and the gradient serves all nb designs
   (so each launch has nb times the parallel work and there are about nb
   times fewer launches per design); the refinement gives each design the
   sweeps its own stopping rule asks for.  APF_FP64 contexts (and GMRES
   refinement) are solved one after the other.  S[b] (may be NULL, or S
   itself NULL), grad_eps[b] (not NULL) and f[b] (host, may be NULL) receive
   design b's results as apf_solve_S_grad would; each context keeps its fields
   for apf_grad_from_gamma.  One stream for all; synchronized before return.
   Returns the first error of any design (APF_ENOCONV: all results
   returned). */
int apf_solve_S_grad_batch(apf_ctx *const *ctx, int nb, int objective, const double *params, int n_params,
                           double *const *S, double *f, double *const *grad_eps, void *stream);

/* df/deps = 2 Re sum_ba Gamma_ba dS_ba/deps for a caller-supplied
   Gamma = df/dS (n_out x n_in complex128), using the fields of the last
   solve (Eq. 1 with Eq. 3).  grad_eps: h*nx float64. */
int apf_grad_from_gamma(apf_ctx *ctx, const double *Gamma, double *grad_eps, void *stream);

/* Orders propagating in the substrate (the reflection channels): *n gets the
   count, m (host, may be NULL) the orders, ascending.  Requires set_grid and
   set_eps. */
int apf_substrate_orders(const apf_ctx *ctx, int *n, int *m);

/* Reflection block of the last solve (paper Sec. 2: S = C A^-1 B - D, with D
   the identity on the reflected channels; Supplement Sec. 1 takes B and C
   from both sides of the structure).  R[b][a] = sqrt(nu_b) u_{m_b}^H E_a on
   the source row minus [m_b == m_a] (the incident wave), for input a and
   substrate order m_ref[b] (host ints, each propagating in the substrate;
   NULL or n_ref = 0: all of apf_substrate_orders).  R: n_ref x n_in
   complex128, [b][a], host or device.  The field on the source row comes
   from the first slab row by the back substitution of the substrate rows,
   per Fourier order.  With lossless permittivity, sum_b |S_ba|^2 over all
   cladding orders plus sum_b |R_ba|^2 over all substrate orders is 1 up to
   the PML reflection (flux conservation).  Enqueues on `stream` and
   synchronizes it. */
int apf_reflection(apf_ctx *ctx, const int *m_ref, int n_ref, double *R, void *stream);

/* Transmission from the cladding side, from the adjoint fields of the last
   solve (A = A^T: the adjoint column of output b is the field of a cladding
   source of order -m_b, scaled by i/2).  S_rev[p][q]: from cladding order
   m_out[q] into substrate order m_in[p], n_in x n_out complex128, [p][q],
   host or device; needs -m in the output set for every output order m
   (APF_EINVAL otherwise; the default channel set qualifies).  Reciprocity
   (paper Sec. 2, dA/dp symmetric) makes S_rev[p(-m_a)][q(-m_b)] = S[b][a]. */
int apf_reverse_S(apf_ctx *ctx, double *S_rev, void *stream);

/* Ridge metasurface parametrization (paper Sec. 3 and Eq. 5: the design
   variables are the edge positions of the ridges; mirror symmetry maps the
   free half period onto the other half, Supplement Sec. 7 frees all edges).
   edges: n_edges float64 (host or device), positions in pixels measured from
   the mirror plane x = nx/2, nondecreasing, ridge i = [t_2i, t_2i+1];
   -nx/2 <= t_0 and t_last <= 0 (mirror != 0) or <= nx/2 (mirror == 0).
   With mirror != 0 the image ridges [-t_2i+1, -t_2i] are added.  Every slab
   row gets the profile eps_x = eps_bg + (eps_ridge - eps_bg) * (length of
   pixel [x, x+1) covered by ridges) -- the paper does not fix the sub-pixel
   treatment; this linear one is continuous in every edge.  The slab is then
   set exactly as apf_set_eps(ctx, eps, j0, h, eps_sub, eps_clad) would;
   eps_out (h*nx, host or device, may be NULL) receives it.  Requires
   apf_set_grid; APF_EINVAL for unsorted, out-of-range or non-finite edges.
   Device-resident edges are read, and eps_out is written, in order on
   `stream` (as for apf_set_eps); the call synchronizes it before returning. */
int apf_set_ridges(apf_ctx *ctx, const double *edges, int n_edges, int mirror,
                   double eps_ridge, double eps_bg, int j0, int h,
                   double eps_sub, double eps_clad, double *eps_out, void *stream);

/* Chain rule from a pixel gradient to the edges of the last apf_set_ridges:
   df/dt_k = sum_{rows, x} (df/deps)[row][x] * deps_x/dt_k, where deps_x/dt_k
   = -+(eps_ridge - eps_bg) on the pixel the edge moves into (minus for a
   ridge's left edge, plus for its right edge) and, with mirror symmetry, on
   the pixel its image moves into (dA/dp_k of rank h, Eq. 2 with r_k = h).
   At an exact pixel boundary the derivative for increasing t is taken.
   grad_eps: h*nx float64 (e.g. from apf_solve_S_grad), grad_edges: n_edges
   float64; host or device each.  Enqueues on `stream` and synchronizes it.
   APF_ESTATE before apf_set_ridges or after the slab was replaced. */
int apf_ridge_grad(apf_ctx *ctx, const double *grad_eps, double *grad_edges, void *stream);

/* Iterative refinement of the mixed mode: stop when max_col ||r||/||R|| <= tol,
   after max_iters sweeps, or when the residual grew on two consecutive sweeps
   (APF_ENOCONV if still above tol).  Defaults: tol 1e-10, max_iters 40.
   Low-contrast slabs need 1-3 sweeps; high-contrast ones (e.g. silicon
   ridges in air) up to ~25 to reach 1e-10. */
int apf_set_refinement(apf_ctx *ctx, double tol, int max_iters);

/* Mixed mode: refine by restarted GMRES(m) instead of plain iterative
   refinement (m = 0, the default).  The low-precision factorization is the
   (right) preconditioner of GMRES, with one Krylov space per right-hand-side
   column; each restart takes m preconditioner applications from the true
   float64 residual, and apf_stats.refine_iters counts those applications.
   It pays on high-contrast slabs, where plain refinement contracts slowly.
   Allocates 2m + 1 field-sized buffers (h x (n_in + n_out) x nx complex128
   each) with the workspace; changing m re-creates the workspace, so the
   fields of an earlier solve are gone.  1 <= m <= 8, or 0. */
int apf_set_krylov(apf_ctx *ctx, int m);

/* Statistics of the last solve: refinement sweeps and residual, device time
   per stage of the pipeline (the stages mirror the paper's breakdown of APF
   time into factorization and post-processing, Supplement Table S1), kernel
   launches and the workspace size.  *stats is written; APF_EINVAL for NULL. */
int apf_get_stats(const apf_ctx *ctx, apf_stats *stats);

/* Mixed mode: storage of the slab Schur blocks.  Every field sweep needs the
   inverses G_j of all h slab rows (the blocks the partial factorization of
   paper Sec. 2 leaves behind; 16 nx^2 bytes each in packed bf16 form, 21.5 GB
   for h = 20 at nx = 8192).  segment_rows = 0 (the default) stores all h.
   segment_rows = k in [1, h) keeps the packed inverses of only one segment of
   k rows, plus the float32 G_{c-1} (8 nx^2 bytes) at every segment start
   c > 0, and recomputes a segment's inverses from its checkpoint whenever a
   sweep needs them: about two eliminations more per sweep, for a workspace
   of (k * 16 + (ceil(h/k) - 1) * 8) nx^2 bytes instead of h * 16 nx^2.  The
   recomputed inverses are bit-identical to the stored ones, so results do
   not change.  Re-creates the workspace like apf_set_krylov (the fields of
   an earlier solve are gone).  APF_EINVAL in APF_FP64 mode for k != 0. */
int apf_set_schur_storage(apf_ctx *ctx, int segment_rows);

/* Mixed mode: accuracy of the low-precision slab elimination (the paper's
   factorization, here an approximate one that float64 refinement corrects).
   planes = 2 (default): every operand is split into two bf16 planes and three
   plane products are summed (bf16x3, about 1e-5 relative per product);
   planes = 3: three planes and six products (bf16x6, about 1e-7), twice the
   tensor work of the elimination and 1.5 times the storage of the packed
   inverses.  High-contrast slabs (e.g. silicon ridges in air) make the slab
   Schur blocks ill-conditioned; their refinement can stall with two planes
   and converges with three.  butterfly = 1 (the mixed-mode default) applies
   a symmetric random butterfly transform (depth 2) to every slab block before
   its inversion (G = U (U^T X U)^-1 U^T), which spreads the rows of strongly
   structured blocks so that the recursion, which pivots only inside its
   32 x 32 leaves, meets no nearly singular leading block: with it the same
   high-contrast slabs converge with two planes, for two memory-bound passes
   over each slab block.  Re-creates the workspace like apf_set_krylov.
   APF_EINVAL for other values, or in APF_FP64 mode for anything but (2, 0). */
int apf_set_elimination(apf_ctx *ctx, int planes, int butterfly);

/* Measurement support (no counterpart in the paper).  When enabled, every
   tensor-core GEMM launch of later solves is bracketed by CUDA events on the
   solve's stream; apf_get_profile returns the totals accumulated since the
   last apf_set_profiling call.  Flops are counted as real multiply-adds x 2:
   alg_flops for the complex products the method needs (8 per complex
   multiply-add), hw_flops for what the tensor pipe executes (alg_flops x the
   number of bf16 plane products). */
typedef struct {
    long long gemm_launches;
    double gemm_ms;
    double gemm_alg_flops;
    double gemm_hw_flops;
} apf_profile;

int apf_set_profiling(apf_ctx *ctx, int enable);
int apf_get_profile(const apf_ctx *ctx, apf_profile *prof);

/* Allocation-free solve for small grids (the paper has no counterpart; it
   exists for callers, not for the method).
   Some callers cannot allocate device memory: code that runs under another
   framework's memory pool, where a direct cudaMalloc would fail or steal
   memory the pool counts on; code with a fixed device-memory budget; code in
   a timing-critical loop, where cudaMalloc's implicit device-wide
   synchronization is not acceptable.  apf_create and the apf_set_* calls
   allocate, so such callers use this one context-free call instead.  It
   computes the same S as apf_create(APF_FP64) + apf_set_grid + apf_set_eps +
   apf_set_channels + apf_solve_S, with the same argument meanings
   (eps_slab: h*nx float64, host or device; m_in / m_out: host int arrays or
   NULL for the default channels; S: n_out*n_in complex128, host or device),
   for nx <= 64 (a power of two), h <= 16 and n_in + n_out <= 128; larger
   problems get APF_EINVAL and a message from apf_last_error(NULL).
   All intermediate arrays live in one file-scope device array of
   APF_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
   holds until the process exits; the call itself never allocates or frees
   device memory.  The first call on a device looks up that array's device
   address (once per device, with the device current); make that first call
   before any stream capture.  The call runs on the current device, enqueues
   on `stream` and synchronizes it before returning.  Every call shares the
   one array and leaves its contents behind (each call zeroes what must start
   at zero); calls on one device take turns like every solve of the library
   (a call blocks on the host while another is inside, see Threads above),
   so calls from several host threads or streams never overlap on it. */
#define APF_NOALLOC_SCRATCH_BYTES (4u << 20)
int apf_solve_S_noalloc(int nx, int ny, int npml_bot, int npml_top, double lambda_px,
                        const apf_pml_params *pml, const double *eps_slab, int j0, int h,
                        double eps_sub, double eps_clad, const int *m_in, int n_in,
                        const int *m_out, int n_out, double *S, void *stream);

/* Message of the most recent failure on this context (or of apf_create when
   ctx is NULL).  Never NULL. */
const char *apf_last_error(const apf_ctx *ctx);

/* ABI version, (major << 16) | minor. */
int apf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* APF_H */
