// Spectral-convolution surrogate of the efficiencies (training and inference
// kernels).  Not part of the paper's method: it screens line-search
// candidates before the exact solve judges them.
//
// Network (x is the periodic axis, n positions; the slab rows are channels):
//   h0 = W0 eps + b0                                   (CI -> C, per position)
//   for l = 1..L:
//     X = DFT_M(h_{l-1})          (first M Fourier modes, e^{-2 pi i m x / n})
//     Y[o, m] = sum_i W_l[i, o, m] X[i, m]             (complex, per mode)
//     z_l = synth_M(Y) + P_l h_{l-1} + c_l              (synth: real inverse DFT
//                                                        of the M modes, zero-padded)
//     h_l = gelu(z_l)  (l < L),   h_L = z_L
//   out = Wh mean_x(h_L) + bh                          (C -> NO)
// Loss: mean squared error.  Weights are used in bf16 (a bf16 copy of the
// fp32 master parameters, refreshed after every Adam step); activations and
// every sum are fp32.
#include "apf_internal.h"
#include "../../include/apf_surrogate.h"

#include <math.h>

#include <vector>

struct apf_sno {
    int device = 0;
    int n = 0, ci = 0, c = 0, m = 0, layers = 0, no = 0, bmax = 0;
    long long nparams = 0;
    // parameter offsets (floats)
    long long oW0, ob0, oWr, oWi, oP, oc, oWh, obh;
    float *p = nullptr, *g = nullptr, *mom1 = nullptr, *mom2 = nullptr;
    __nv_bfloat16 *pb = nullptr;
    float2 *tw = nullptr;          // M x n: (cos, sin)(2 pi m x / n)
    float *h = nullptr, *z = nullptr;       // (L+1) x B x C x n, L x B x C x n
    float2 *X = nullptr, *Y = nullptr;      // L x B x C x M
    float *dh = nullptr, *dhp = nullptr, *dz = nullptr;  // B x C x n each
    float2 *dY = nullptr, *dX = nullptr;    // B x C x M
    float *pooled = nullptr, *out = nullptr, *dout = nullptr, *dpooled = nullptr, *loss = nullptr;
    long long step = 0;
    std::vector<void *> allocs;
    std::string err;
};

namespace {

__device__ __forceinline__ float bf(const __nv_bfloat16 *p, long long i) { return __bfloat162float(p[i]); }

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    const float phi = 0.39894228040143268f * expf(-0.5f * x * x);
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * phi;
}

__global__ void k_tw(float2 *tw, int n, int M) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (x >= n) return;
    long long t = ((long long)m * x) % n;
    float s, c;
    sincospif(2.f * (float)t / (float)n, &s, &c);
    tw[(long long)m * n + x] = make_float2(c, s);
}

// h0[b][o][x] = b0[o] + sum_i W0[o][i] eps[b][i][x]
__global__ void k_lift(const float *eps, const __nv_bfloat16 *pb, long long oW0, long long ob0, float *h0, int B,
                       int CI, int C, int n) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)B * C * n;
    if (idx >= total) return;
    int x = idx % n;
    int o = (idx / n) % C;
    int b = idx / ((long long)n * C);
    float acc = bf(pb, ob0 + o);
    for (int i = 0; i < CI; ++i) acc += bf(pb, oW0 + (long long)o * CI + i) * eps[((long long)b * CI + i) * n + x];
    h0[idx] = acc;
}

// out[row][m] = scale_m * sum_x in[row][x] (cos, -sin)(theta_mx), rows = B*C.
// scale_m = 1 (analysis) or the synthesis weights (1/n, 2/n) for the backward.
__global__ void k_dft(const float *in, float2 *out, const float2 *tw, int n, int M, int synth_weights) {
    extern __shared__ float row[];
    const long long r = blockIdx.x;
    for (int x = threadIdx.x; x < n; x += blockDim.x) row[x] = in[r * n + x];
    __syncthreads();
    // 4 threads per mode
    const int m = threadIdx.x >> 2, part = threadIdx.x & 3;
    float ar = 0.f, ai = 0.f;
    if (m < M) {
        const float2 *t = tw + (long long)m * n;
        for (int x = part; x < n; x += 4) {
            float v = row[x];
            float2 w = t[x];
            ar += v * w.x;
            ai -= v * w.y;
        }
    }
    ar += __shfl_xor_sync(0xffffffffu, ar, 1);
    ai += __shfl_xor_sync(0xffffffffu, ai, 1);
    ar += __shfl_xor_sync(0xffffffffu, ar, 2);
    ai += __shfl_xor_sync(0xffffffffu, ai, 2);
    if (m < M && part == 0) {
        float s = 1.f;
        if (synth_weights) s = (m == 0 ? 1.f : 2.f) / (float)n;
        out[r * M + m] = make_float2(ar * s, ai * s);
    }
}

// Y[b][o][m] = sum_i W[i][o][m] X[b][i][m]
__global__ void k_mix(const float2 *X, const __nv_bfloat16 *pb, long long oWr, long long oWi, float2 *Y, int B, int C,
                      int M) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)B * C * M) return;
    int m = idx % M;
    int o = (idx / M) % C;
    int b = idx / ((long long)M * C);
    float yr = 0.f, yi = 0.f;
    for (int i = 0; i < C; ++i) {
        float2 x = X[((long long)b * C + i) * M + m];
        long long wi = ((long long)i * C + o) * M + m;
        float wr = bf(pb, oWr + wi), wim = bf(pb, oWi + wi);
        yr += wr * x.x - wim * x.y;
        yi += wr * x.y + wim * x.x;
    }
    Y[idx] = make_float2(yr, yi);
}

// z[b][o][x] = sum_m w_m Re(Y e^{i theta}) + sum_i P[o][i] h[b][i][x] + c[o];  hn = act(z)
__global__ void k_synth(const float2 *Y, const float *h, const __nv_bfloat16 *pb, long long oP, long long oc,
                        const float2 *tw, float *z, float *hn, int C, int n, int M, int act) {
    extern __shared__ float sm[];
    float2 *ys = reinterpret_cast<float2 *>(sm);  // M
    float *ps = sm + 2 * M;                         // C
    const int bo = blockIdx.y;                      // b * C + o
    const int b = bo / C, o = bo % C;
    for (int m = threadIdx.x; m < M; m += blockDim.x) ys[m] = Y[(long long)bo * M + m];
    for (int i = threadIdx.x; i < C; i += blockDim.x) ps[i] = bf(pb, oP + (long long)o * C + i);
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    float acc = 0.f;
    for (int m = 0; m < M; ++m) {
        float2 w = tw[(long long)m * n + x];
        float2 y = ys[m];
        float s = (m == 0 ? 1.f : 2.f) / (float)n;
        acc += s * (y.x * w.x - y.y * w.y);
    }
    for (int i = 0; i < C; ++i) acc += ps[i] * h[((long long)b * C + i) * n + x];
    acc += bf(pb, oc + o);
    long long idx = (long long)bo * n + x;
    z[idx] = acc;
    hn[idx] = act ? gelu(acc) : acc;
}

// pooled[b][c] = mean_x h[b][c][x]
__global__ void k_pool(const float *h, float *pooled, int n) {
    __shared__ float red[256];
    const long long r = blockIdx.x;
    float acc = 0.f;
    for (int x = threadIdx.x; x < n; x += blockDim.x) acc += h[r * n + x];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) pooled[r] = red[0] / (float)n;
}

__global__ void k_head(const float *pooled, const __nv_bfloat16 *pb, long long oWh, long long obh, float *out, int B,
                       int C, int NO) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * NO) return;
    int k = idx % NO, b = idx / NO;
    float acc = bf(pb, obh + k);
    for (int c = 0; c < C; ++c) acc += bf(pb, oWh + (long long)k * C + c) * pooled[(long long)b * C + c];
    out[idx] = acc;
}

// Loss, d_out, head gradients and d_pooled (one block).
__global__ void k_head_bwd(const float *out, const float *tgt, const float *pooled, const __nv_bfloat16 *pb,
                           long long oWh, float *g, long long gWh, long long gbh, float *dout, float *dpooled,
                           float *loss, int B, int C, int NO) {
    __shared__ float red[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < B * NO; i += blockDim.x) {
        float d = out[i] - tgt[i];
        acc += d * d;
        dout[i] = 2.f * d / (float)(B * NO);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = red[0] / (float)(B * NO);
    for (int e = threadIdx.x; e < NO * C; e += blockDim.x) {
        int k = e / C, c = e % C;
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dout[b * NO + k] * pooled[(long long)b * C + c];
        g[gWh + e] = s;
    }
    for (int k = threadIdx.x; k < NO; k += blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dout[b * NO + k];
        g[gbh + k] = s;
    }
    for (int e = threadIdx.x; e < B * C; e += blockDim.x) {
        int b = e / C, c = e % C;
        float s = 0.f;
        for (int k = 0; k < NO; ++k) s += dout[b * NO + k] * bf(pb, oWh + (long long)k * C + c);
        dpooled[e] = s;
    }
}

// dz = dh * act'(z)  (dh of the last layer is the broadcast of dpooled / n)
__global__ void k_act_bwd(const float *dh, const float *dpooled, const float *z, float *dz, long long total, int n,
                          int act) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    float d = dpooled ? dpooled[i / n] / (float)n : dh[i];
    dz[i] = act ? d * gelu_d(z[i]) : d;
}

// G[o][i] += sum_{b,x} D[b][o][x] H[b][i][x] and gc[o] += sum D  (one block per batch
// sample, x staged in chunks of 64, fp32 atomics into the gradient)
__global__ void k_outer(const float *D, const float *H, float *G, float *gc, int CO, int CI, int n) {
    extern __shared__ float sm[];
    float *ds = sm;             // CO x 64
    float *hs = sm + CO * 64;   // CI x 64
    const int b = blockIdx.x;
    const int pairs = CO * CI;
    float acc[12];
    float cacc = 0.f;
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = 0.f;
    for (int x0 = 0; x0 < n; x0 += 64) {
        for (int e = threadIdx.x; e < CO * 64; e += blockDim.x)
            ds[e] = D[((long long)b * CO + e / 64) * n + x0 + (e % 64)];
        for (int e = threadIdx.x; e < CI * 64; e += blockDim.x)
            hs[e] = H[((long long)b * CI + e / 64) * n + x0 + (e % 64)];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            int pr = threadIdx.x + q * blockDim.x;
            if (pr < pairs) {
                int o = pr / CI, i = pr % CI;
                float s = 0.f;
                for (int x = 0; x < 64; ++x) s += ds[o * 64 + x] * hs[i * 64 + x];
                acc[q] += s;
            }
        }
        if (gc && (int)threadIdx.x < CO)
            for (int x = 0; x < 64; ++x) cacc += ds[threadIdx.x * 64 + x];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        int pr = threadIdx.x + q * blockDim.x;
        if (pr < pairs) atomicAdd(&G[pr], acc[q]);
    }
    if (gc && (int)threadIdx.x < CO) atomicAdd(&gc[threadIdx.x], cacc);
}

// Mixing backward: dX[b][i][m] = sum_o conj-pair(W) dY;  dW[i][o][m] = sum_b ...
__global__ void k_mix_bwd_x(const float2 *dY, const __nv_bfloat16 *pb, long long oWr, long long oWi, float2 *dX, int B,
                            int C, int M) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)B * C * M) return;
    int m = idx % M;
    int i = (idx / M) % C;
    int b = idx / ((long long)M * C);
    float xr = 0.f, xi = 0.f;
    for (int o = 0; o < C; ++o) {
        float2 d = dY[((long long)b * C + o) * M + m];
        long long wi = ((long long)i * C + o) * M + m;
        float wr = bf(pb, oWr + wi), wim = bf(pb, oWi + wi);
        xr += wr * d.x + wim * d.y;
        xi += -wim * d.x + wr * d.y;
    }
    dX[idx] = make_float2(xr, xi);
}

__global__ void k_mix_bwd_w(const float2 *X, const float2 *dY, float *g, long long gWr, long long gWi, int B, int C,
                            int M) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)C * C * M) return;
    int m = idx % M;
    int o = (idx / M) % C;
    int i = idx / ((long long)M * C);
    float ar = 0.f, ai = 0.f;
    for (int b = 0; b < B; ++b) {
        float2 x = X[((long long)b * C + i) * M + m];
        float2 d = dY[((long long)b * C + o) * M + m];
        ar += x.x * d.x + x.y * d.y;
        ai += -x.y * d.x + x.x * d.y;
    }
    g[gWr + idx] = ar;
    g[gWi + idx] = ai;
}

// dh_prev[b][i][x] = sum_o P[o][i] dz[b][o][x] + sum_m (dXr cos - dXi sin)
__global__ void k_dh_prev(const float *dz, const float2 *dX, const __nv_bfloat16 *pb, long long oP, const float2 *tw,
                          float *dhp, int C, int n, int M) {
    extern __shared__ float sm[];
    float2 *xs = reinterpret_cast<float2 *>(sm);
    float *ps = sm + 2 * M;
    const int bi = blockIdx.y;
    const int b = bi / C, i = bi % C;
    for (int m = threadIdx.x; m < M; m += blockDim.x) xs[m] = dX[(long long)bi * M + m];
    for (int o = threadIdx.x; o < C; o += blockDim.x) ps[o] = bf(pb, oP + (long long)o * C + i);
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    float acc = 0.f;
    for (int o = 0; o < C; ++o) acc += ps[o] * dz[((long long)b * C + o) * n + x];
    for (int m = 0; m < M; ++m) {
        float2 w = tw[(long long)m * n + x];
        float2 d = xs[m];
        acc += d.x * w.x - d.y * w.y;
    }
    dhp[(long long)bi * n + x] = acc;
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, __nv_bfloat16 *pb, long long np, float lr,
                       float b1, float b2, float c1, float c2, float epsv) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float a = b1 * m1[i] + (1.f - b1) * gi;
    float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    float q = p[i] - lr * (a / c1) / (sqrtf(v / c2) + epsv);
    p[i] = q;
    pb[i] = __float2bfloat16_rn(q);
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *pb, long long np) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < np) pb[i] = __float2bfloat16_rn(p[i]);
}

unsigned nb(long long total, int t = 256) { return (unsigned)((total + t - 1) / t); }

int serr(apf_sno *s, int code, const char *msg) {
    if (s) s->err = msg;
    return set_err(nullptr, code, "%s", msg);
}

void forward(apf_sno *s, const float *x, int B, cudaStream_t st) {
    const int C = s->c, n = s->n, M = s->m, L = s->layers;
    const long long act = (long long)B * C * n, spec = (long long)B * C * M;
    k_lift<<<nb(act), 256, 0, st>>>(x, s->pb, s->oW0, s->ob0, s->h, B, s->ci, C, n);
    for (int l = 0; l < L; ++l) {
        const float *hp = s->h + (long long)l * s->bmax * C * n;
        float *hn = s->h + (long long)(l + 1) * s->bmax * C * n;
        float *z = s->z + (long long)l * s->bmax * C * n;
        float2 *X = s->X + (long long)l * s->bmax * C * M, *Y = s->Y + (long long)l * s->bmax * C * M;
        k_dft<<<B * C, 4 * M, n * sizeof(float), st>>>(hp, X, s->tw, n, M, 0);
        k_mix<<<nb(spec), 256, 0, st>>>(X, s->pb, s->oWr + (long long)l * C * C * M, s->oWi + (long long)l * C * C * M,
                                       Y, B, C, M);
        dim3 g((n + 255) / 256, B * C);
        k_synth<<<g, 256, (2 * M + C) * sizeof(float), st>>>(Y, hp, s->pb, s->oP + (long long)l * C * C,
                                                           s->oc + (long long)l * C, s->tw, z, hn, C, n, M,
                                                           l < L - 1 ? 1 : 0);
    }
    (void)act;
    k_pool<<<B * C, 256, 0, st>>>(s->h + (long long)L * s->bmax * C * n, s->pooled, n);
    k_head<<<nb(B * s->no), 256, 0, st>>>(s->pooled, s->pb, s->oWh, s->obh, s->out, B, C, s->no);
}

// Gradients of the loss w.r.t. every parameter into s->g (after forward).
void backward(apf_sno *s, const float *x, const float *tgt, int B, cudaStream_t st) {
    const int C = s->c, n = s->n, M = s->m, L = s->layers, NO = s->no;
    const long long act = (long long)B * C * n, spec = (long long)B * C * M;
    cudaMemsetAsync(s->g, 0, sizeof(float) * s->nparams, st);
    k_head_bwd<<<1, 256, 0, st>>>(s->out, tgt, s->pooled, s->pb, s->oWh, s->g, s->oWh, s->obh, s->dout, s->dpooled,
                                  s->loss, B, C, NO);
    for (int l = L - 1; l >= 0; --l) {
        const float *hp = s->h + (long long)l * s->bmax * C * n;
        const float *z = s->z + (long long)l * s->bmax * C * n;
        const float2 *X = s->X + (long long)l * s->bmax * C * M;
        k_act_bwd<<<nb(act), 256, 0, st>>>(s->dh, l == L - 1 ? s->dpooled : nullptr, z, s->dz, act, n,
                                           l < L - 1 ? 1 : 0);
        k_outer<<<B, 256, (C + C) * 64 * sizeof(float), st>>>(s->dz, hp, s->g + s->oP + (long long)l * C * C,
                                                             s->g + s->oc + (long long)l * C, C, C, n);
        k_dft<<<B * C, 4 * M, n * sizeof(float), st>>>(s->dz, s->dY, s->tw, n, M, 1);
        k_mix_bwd_w<<<nb((long long)C * C * M), 256, 0, st>>>(X, s->dY, s->g, s->oWr + (long long)l * C * C * M,
                                                              s->oWi + (long long)l * C * C * M, B, C, M);
        k_mix_bwd_x<<<nb(spec), 256, 0, st>>>(s->dY, s->pb, s->oWr + (long long)l * C * C * M,
                                              s->oWi + (long long)l * C * C * M, s->dX, B, C, M);
        dim3 g((n + 255) / 256, B * C);
        k_dh_prev<<<g, 256, (2 * M + C) * sizeof(float), st>>>(s->dz, s->dX, s->pb, s->oP + (long long)l * C * C,
                                                             s->tw, s->dhp, C, n, M);
        float *t = s->dh;
        s->dh = s->dhp;
        s->dhp = t;
    }
    // lift: dW0[o][i] = sum dh0[b][o][x] eps[b][i][x], db0 = sum dh0
    k_outer<<<B, 256, (C + s->ci) * 64 * sizeof(float), st>>>(s->dh, x, s->g + s->oW0, s->g + s->ob0, C, s->ci, n);
}

}  // namespace

extern "C" {

int apf_sno_create(apf_sno **out, int device, int n, int in_ch, int width, int modes, int layers, int n_out,
                   int max_batch) {
    if (!out) return APF_EINVAL;
    *out = nullptr;
    if (n < 64 || (n % 64) || in_ch < 1 || in_ch > 64 || width < 1 || width > 64 || modes < 1 || 2 * modes > n ||
        modes > 256 || layers < 1 || layers > 8 || n_out < 1 || n_out > 64 || max_batch < 1 || max_batch > 4096 ||
        width * width > 12 * 256 || width * in_ch > 12 * 256)
        return set_err(nullptr, APF_EINVAL, "apf_sno_create: sizes out of range");
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return set_err(nullptr, APF_ECUDA, "bad device"); }
    apf_sno *s = new apf_sno();
    s->device = device; s->n = n; s->ci = in_ch; s->c = width; s->m = modes; s->layers = layers; s->no = n_out;
    s->bmax = max_batch;
    const long long C = width, M = modes, L = layers;
    long long o = 0;
    s->oW0 = o; o += C * in_ch;
    s->ob0 = o; o += C;
    s->oWr = o; o += L * C * C * M;
    s->oWi = o; o += L * C * C * M;
    s->oP = o; o += L * C * C;
    s->oc = o; o += L * C;
    s->oWh = o; o += (long long)n_out * C;
    s->obh = o; o += n_out;
    s->nparams = o;
    const long long Bn = (long long)max_batch * C * n, BM = (long long)max_batch * C * M;
    auto al = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        s->allocs.push_back(*p);
        return true;
    };
    bool ok = al((void **)&s->p, sizeof(float) * o) && al((void **)&s->g, sizeof(float) * o) &&
              al((void **)&s->mom1, sizeof(float) * o) && al((void **)&s->mom2, sizeof(float) * o) &&
              al((void **)&s->pb, sizeof(__nv_bfloat16) * o) && al((void **)&s->tw, sizeof(float2) * M * n) &&
              al((void **)&s->h, sizeof(float) * (L + 1) * Bn) && al((void **)&s->z, sizeof(float) * L * Bn) &&
              al((void **)&s->X, sizeof(float2) * L * BM) && al((void **)&s->Y, sizeof(float2) * L * BM) &&
              al((void **)&s->dh, sizeof(float) * Bn) && al((void **)&s->dhp, sizeof(float) * Bn) &&
              al((void **)&s->dz, sizeof(float) * Bn) && al((void **)&s->dY, sizeof(float2) * BM) &&
              al((void **)&s->dX, sizeof(float2) * BM) &&
              al((void **)&s->pooled, sizeof(float) * max_batch * C) &&
              al((void **)&s->dpooled, sizeof(float) * max_batch * C) &&
              al((void **)&s->out, sizeof(float) * max_batch * n_out) &&
              al((void **)&s->dout, sizeof(float) * max_batch * n_out) && al((void **)&s->loss, sizeof(float) * 4);
    if (!ok) {
        cudaGetLastError();
        apf_sno_destroy(s);
        return set_err(nullptr, APF_ENOMEM, "apf_sno_create: out of device memory");
    }
    cudaMemset(s->p, 0, sizeof(float) * o);
    cudaMemset(s->mom1, 0, sizeof(float) * o);
    cudaMemset(s->mom2, 0, sizeof(float) * o);
    k_tw<<<dim3((n + 255) / 256, modes), 256>>>(s->tw, n, modes);
    k_to_bf16<<<nb(o), 256>>>(s->p, s->pb, o);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        apf_sno_destroy(s);
        return set_err(nullptr, APF_ECUDA, "apf_sno_create: init failed");
    }
    *out = s;
    return APF_OK;
}

void apf_sno_destroy(apf_sno *s) {
    if (!s) return;
    cudaSetDevice(s->device);
    for (void *p : s->allocs) cudaFree(p);
    delete s;
}

long long apf_sno_num_params(const apf_sno *s) { return s ? s->nparams : -1; }

int apf_sno_set_params(apf_sno *s, const float *params) {
    if (!s || !params) return APF_EINVAL;
    cudaSetDevice(s->device);
    if (cudaMemcpy(s->p, params, sizeof(float) * s->nparams, cudaMemcpyDefault) != cudaSuccess)
        return serr(s, APF_ECUDA, "set_params copy failed");
    cudaMemset(s->mom1, 0, sizeof(float) * s->nparams);
    cudaMemset(s->mom2, 0, sizeof(float) * s->nparams);
    s->step = 0;
    k_to_bf16<<<nb(s->nparams), 256>>>(s->p, s->pb, s->nparams);
    return cudaDeviceSynchronize() == cudaSuccess ? APF_OK : serr(s, APF_ECUDA, "set_params failed");
}

int apf_sno_get_params(const apf_sno *s, float *params) {
    if (!s || !params) return APF_EINVAL;
    cudaSetDevice(s->device);
    return cudaMemcpy(params, s->p, sizeof(float) * s->nparams, cudaMemcpyDefault) == cudaSuccess ? APF_OK
                                                                                                  : APF_ECUDA;
}

int apf_sno_forward(apf_sno *s, const float *x, int B, float *y, void *stream) {
    if (!s || !x || !y || B < 1 || B > s->bmax) return APF_EINVAL;
    cudaSetDevice(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    forward(s, x, B, st);
    cudaMemcpyAsync(y, s->out, sizeof(float) * B * s->no, cudaMemcpyDefault, st);
    cudaError_t e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? APF_OK : serr(s, APF_ECUDA, cudaGetErrorString(e));
}

int apf_sno_gradients(apf_sno *s, const float *x, const float *target, int B, float *grads, float *loss,
                      void *stream) {
    if (!s || !x || !target || B < 1 || B > s->bmax) return APF_EINVAL;
    cudaSetDevice(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    forward(s, x, B, st);
    backward(s, x, target, B, st);
    if (grads) cudaMemcpyAsync(grads, s->g, sizeof(float) * s->nparams, cudaMemcpyDefault, st);
    float lh = 0.f;
    cudaMemcpyAsync(&lh, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (loss) *loss = lh;
    return e == cudaSuccess ? APF_OK : serr(s, APF_ECUDA, cudaGetErrorString(e));
}

int apf_sno_train_step(apf_sno *s, const float *x, const float *target, int B, float lr, float *loss,
                       void *stream) {
    if (!s || !x || !target || B < 1 || B > s->bmax || !(lr > 0.f)) return APF_EINVAL;
    cudaSetDevice(s->device);
    cudaStream_t st = (cudaStream_t)stream;
    forward(s, x, B, st);
    backward(s, x, target, B, st);
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)s->step), c2 = 1.f - powf(b2, (float)s->step);
    k_adam<<<nb(s->nparams), 256, 0, st>>>(s->p, s->g, s->mom1, s->mom2, s->pb, s->nparams, lr, b1, b2, c1, c2,
                                           1e-8f);
    float lh = 0.f;
    cudaMemcpyAsync(&lh, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (loss) *loss = lh;
    return e == cudaSuccess ? APF_OK : serr(s, APF_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
