/*
 * apf_surrogate.h -- C ABI of the spectral-convolution surrogate.
 *
 * The paper has no learned component: this network exists to screen many
 * candidate line-search steps (Supplement Sec. 4, backtracking with the
 * Armijo condition of Eq. S2) cheaply; the exact solve (apf.h) still judges
 * and accepts every step.  It maps the slab permittivity (in_ch slab rows as
 * channels, n periodic positions) to n_out numbers (here the efficiencies of
 * the relative diffraction orders -2..2, averaged over the inputs).
 *
 * Network: lift (in_ch -> width per position), `layers` spectral layers
 * (truncated DFT to `modes` modes, per-mode complex width x width mixing,
 * real inverse DFT, plus a per-position width x width map and bias; GELU on
 * all but the last), mean over positions, linear head (width -> n_out).
 * Weights are applied in bf16 (a copy of the fp32 master parameters, refreshed
 * after every Adam step); activations and all sums are fp32.
 *
 * Parameter vector (fp32, flat, in this order): W0[width][in_ch], b0[width],
 * Wr[layers][width_in][width_out][modes], Wi[...same...], P[layers][width][width]
 * ([out][in]), c[layers][width], Wh[n_out][width], bh[n_out].
 *
 * Arrays: x is batch x in_ch x n fp32 (row-major), targets / outputs batch x
 * n_out fp32; host or device pointers.  Calls enqueue on `stream` and
 * synchronize it before returning.  Return codes as in apf.h; errors are
 * described by apf_last_error(NULL).  The handle owns its device memory
 * (allocated by apf_sno_create only).
 */
#ifndef APF_SURROGATE_H
#define APF_SURROGATE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apf_sno apf_sno;

/* n a multiple of 64 with 2*modes <= n; width <= 64; in_ch <= 64; layers <= 8;
   max_batch <= 4096.  Parameters start at zero: set them with apf_sno_set_params. */
int apf_sno_create(apf_sno **out, int device, int n, int in_ch, int width, int modes, int layers,
                   int n_out, int max_batch);
void apf_sno_destroy(apf_sno *s);
long long apf_sno_num_params(const apf_sno *s);
/* Copy the fp32 parameters in (also resets the Adam moments) or out. */
int apf_sno_set_params(apf_sno *s, const float *params);
int apf_sno_get_params(const apf_sno *s, float *params);
/* y = net(x) for `batch` samples. */
int apf_sno_forward(apf_sno *s, const float *x, int batch, float *y, void *stream);
/* Gradient of the mean squared error w.r.t. every parameter (same layout as
   the parameter vector; grads may be NULL) and the loss (host, may be NULL). */
int apf_sno_gradients(apf_sno *s, const float *x, const float *target, int batch, float *grads,
                      float *loss, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error. */
int apf_sno_train_step(apf_sno *s, const float *x, const float *target, int batch, float lr,
                       float *loss, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* APF_SURROGATE_H */
