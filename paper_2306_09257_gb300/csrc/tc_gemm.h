// Tensor-core GEMM interface (internal).
#pragma once
#include "apf_internal.h"

#include <cuda.h>

// A packed bf16 operand: `planes` split planes of `rows` rows, each row
// `kp` bf16 values (kp a multiple of 64); plane p row r at
// base + p * plane_pitch + r * kp.
struct PackView {
    const __nv_bfloat16 *base;
    long long rows;
    long long kp;
    int planes;
    long long plane_pitch;
};

struct TcParams {
    int M, N, n_cplx;
    int kblocks, nseg;
    uint32_t seg_pairs;
    float alpha, beta;
    float *out_re, *out_im;
    long long ldo;
    const float *in_re, *in_im;
    long long ldi;
    int *flags;
};

// Up to P products of the same shape in one launch (the designs of a batch):
// per problem its two operand tensor maps and its output/input planes.
template <int P>
struct TcArgs {
    CUtensorMap a[P], b[P];
    TcParams p[P];
    int nprob;
};
constexpr int TC_MAX_BATCH = 16;

// One product of a batch: operands, output (and beta input) planes, error flags.
struct TcProblem {
    PackView A, B;
    float *out_re, *out_im;
    const float *in_re, *in_im;
    int *flags;
};

uint32_t tc_seg_pairs(int nsplit, int *nseg);
void tc_init_attrs();

// out = alpha * (A B^T) + beta * in, where output column col < n_cplx goes to
// the real plane (column col) and col >= n_cplx to the imaginary plane
// (column col - n_cplx).  A: M rows; B: N rows; both with the same kp.
int tc_gemm(apf_ctx *c, const PackView &A, const PackView &B, int nsplit, int M, int N, int n_cplx, float alpha,
            float beta, float *out_re, float *out_im, long long ldo, const float *in_re, const float *in_im,
            long long ldi, cudaStream_t s);
// nprob (<= TC_MAX_BATCH) products of the same shape in one launch.
int tc_gemm_n(apf_ctx *c, int nprob, const TcProblem *pb, int nsplit, int M, int N, int n_cplx, float alpha,
              float beta, long long ldo, long long ldi, cudaStream_t s);
