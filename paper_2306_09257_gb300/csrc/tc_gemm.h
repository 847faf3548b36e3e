// Tensor-core GEMM interface (internal).
#pragma once
#include "apf_internal.h"

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
    // optional extra outputs of the same value v = alpha * acc + beta * in
    // (output row r, complex column c; `re` for col < n_cplx, `im` otherwise):
    float *t_re, *t_im;      // transposed fp32: t[c][r]
    long long ldt;
    int pk_nsplit;           // bf16 planes of the packs below
    __nv_bfloat16 *pkA;      // A-layout pack of the rows: plane p, row r, position col
    long long pkA_kp, pkA_pitch;
    __nv_bfloat16 *pkBT;     // B-layout pack of the transpose (rows c and n_cplx + c, k = r)
    long long pkBT_kp, pkBT_pitch;
    __nv_bfloat16 *pkAT;     // A-layout pack of the transpose (row c, k = r / M + r)
    long long pkAT_kp, pkAT_pitch;
    int kM;                  // M as the k extent of the transposed packs
};

// Extra epilogue outputs for tc_gemm_ex.
struct TcSinks {
    float *t_re = nullptr, *t_im = nullptr;
    long long ldt = 0;
    bool skip_fp32 = false;  // do not write the row-major fp32 output
    int nsplit = 2;
    __nv_bfloat16 *pkA = nullptr;
    long long pkA_kp = 0, pkA_pitch = 0;
    __nv_bfloat16 *pkBT = nullptr;
    long long pkBT_kp = 0, pkBT_pitch = 0;
    __nv_bfloat16 *pkAT = nullptr;
    long long pkAT_kp = 0, pkAT_pitch = 0;
};

uint32_t tc_seg_pairs(int nsplit, int *nseg);
void tc_init_attrs();

// out = alpha * (A B^T) + beta * in, where output column col < n_cplx goes to
// the real plane (column col) and col >= n_cplx to the imaginary plane
// (column col - n_cplx).  A: M rows; B: N rows; both with the same kp.
int tc_gemm(apf_ctx *c, const PackView &A, const PackView &B, int nsplit, int M, int N, int n_cplx, float alpha,
            float beta, float *out_re, float *out_im, long long ldo, const float *in_re, const float *in_im,
            long long ldi, cudaStream_t s);
int tc_gemm_ex(apf_ctx *c, const PackView &A, const PackView &B, int nsplit, int M, int N, int n_cplx, float alpha,
               float beta, float *out_re, float *out_im, long long ldo, const float *in_re, const float *in_im,
               long long ldi, const TcSinks &sk, cudaStream_t s);
