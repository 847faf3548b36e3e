// Tensor-core GEMM for sm_103a: tcgen05.mma (kind::f16, bf16 operands, fp32
// accumulation in tensor memory), operands staged by TMA with 128-byte
// swizzle, warp-specialized (1 TMA producer warp, 1 MMA-issuing warp, 4
// epilogue warps).
//
// The GEMM is real: D[m][n] = sum_k A[m][k] B[n][k] with A and B "K-major"
// (rows contiguous in k).  Complex products and extra precision are both
// expressed through the operand layout, so one real kernel serves all of the
// slab elimination:
//   * complex: A-row = [Re a, Im a], B-rows = [Re b, -Im b] (real part of the
//     output) and [Im b, Re b] (imaginary part), so a complex m x k x n product
//     is one real m x 2k x 2n product;
//   * precision: each operand is split into 2 or 3 bf16 planes
//     (x = x0 + x1 [+ x2]); the kernel walks "segments", one per retained
//     plane product (x0 y0, x0 y1, x1 y0 [, x0 y2, x1 y1, x2 y0]), all
//     accumulated in the same fp32 tensor-memory tile.
// Operand planes live in 3-D tensor maps (k, row, plane), so rows past the
// operand's end are zero-filled by TMA and no padding is needed in m or n.
#include "apf_internal.h"
#include "tc_gemm.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <stdlib.h>
#include <string.h>

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // bf16 elements per 128-byte swizzle row

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^31 clock cycles (about a second) or when
// another role of this block has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          bool ignore_abort = false) {
    long long t0 = clock64();
    uint32_t spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 1023u) == 0) {
            if (!ignore_abort && *abort_flag) return false;
            if (clock64() - t0 > (1ll << 31)) return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(smem_dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms of 1024 bytes (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int BN, int STAGES>
struct Layout {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR = STAGES * STAGE;
    static constexpr int TOTAL = BAR + (2 * STAGES + 4) * 8 + 16 + 1024;
};

// Epilogue of one 32-column chunk of one accumulator row.
__device__ __forceinline__ void store_chunk(const TcParams &p, int row, int col0, const uint32_t (&r)[32]) {
    if (row >= p.M) return;
    const bool use_beta = (p.beta != 0.0f);
    float *op;
    const float *ip;
    int cc0;
    if (col0 < p.n_cplx) { op = p.out_re; ip = p.in_re; cc0 = col0; }
    else { op = p.out_im; ip = p.in_im; cc0 = col0 - p.n_cplx; }
    const bool whole = (col0 + 32 <= p.N) && ((col0 < p.n_cplx) == (col0 + 31 < p.n_cplx));
    float *dst = op + (long long)row * p.ldo + cc0;
    const float *src = ip + (long long)row * p.ldi + cc0;
    if (whole && ((((uintptr_t)dst) | (use_beta ? (uintptr_t)src : 0)) & 15) == 0) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            float4 o;
            o.x = p.alpha * __uint_as_float(r[4 * v + 0]);
            o.y = p.alpha * __uint_as_float(r[4 * v + 1]);
            o.z = p.alpha * __uint_as_float(r[4 * v + 2]);
            o.w = p.alpha * __uint_as_float(r[4 * v + 3]);
            if (use_beta) {
                float4 c = *reinterpret_cast<const float4 *>(src + 4 * v);
                o.x += p.beta * c.x; o.y += p.beta * c.y; o.z += p.beta * c.z; o.w += p.beta * c.w;
            }
            *reinterpret_cast<float4 *>(dst + 4 * v) = o;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int col = col0 + i;
        if (col >= p.N) break;
        float *o2;
        const float *i2;
        int cc;
        if (col < p.n_cplx) { o2 = p.out_re; i2 = p.in_re; cc = col; }
        else { o2 = p.out_im; i2 = p.in_im; cc = col - p.n_cplx; }
        float v = p.alpha * __uint_as_float(r[i]);
        if (use_beta) v += p.beta * i2[(long long)row * p.ldi + cc];
        o2[(long long)row * p.ldo + cc] = v;
    }
}

// Persistent: one CTA per SM walks the output tiles (M index fastest, so the
// CTAs working on one B panel run together); two tensor-memory accumulators
// let the epilogue of one tile overlap the MMAs of the next.
template <int BN, int STAGES, int P>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ TcArgs<P> args) {
    using L = Layout<BN, STAGES>;
    const TcParams &p = args.p[0];  // shape and precision: the same for every problem
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + L::BAR);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;   // [2]
    uint64_t *tempty = tfull + 2;       // [2]
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Mt = (p.M + BM - 1) / BM, Nt = (p.N + BN - 1) / BN;
    const int ntl = Mt * Nt, ntiles = ntl * args.nprob;  // tiles of problem pr: [pr ntl, (pr + 1) ntl)
    const int total = p.nseg * p.kblocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    int issued = 0;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int pr = tile / ntl, tt = tile - pr * ntl;
                const int m0 = (tt % Mt) * BM, n0 = (tt / Mt) * BN;
                const CUtensorMap *tmA = &args.a[pr], *tmB = &args.b[pr];
                for (int kk = 0; kk < total; ++kk, ++it) {
                    const int s = it % STAGES, r = it / STAGES;
                    if (!mbar_wait(&empty[s], (r & 1) ^ 1, abort_flag)) { ok = false; break; }
                    const int seg = kk / p.kblocks, kb = kk - seg * p.kblocks;
                    const int pa = (p.seg_pairs >> (4 * seg + 2)) & 3, pb = (p.seg_pairs >> (4 * seg)) & 3;
                    uint8_t *sa = smem + s * L::STAGE;
                    uint8_t *sb = sa + L::A_BYTES;
                    mbar_expect_tx(&full[s], L::A_BYTES + L::B_BYTES);
                    tma_load_3d(sa, tmA, &full[s], kb * BK, m0, pa);
                    tma_load_3d(sb, tmB, &full[s], kb * BK, n0, pb);
                    issued = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
            int it = 0, tl = 0;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tl) {
                const int b = tl & 1, u = tl >> 1;
                if (!mbar_wait(&tempty[b], (u & 1) ^ 1, abort_flag)) { ok = false; break; }
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * BN);
                for (int kk = 0; kk < total; ++kk, ++it) {
                    const int s = it % STAGES, r = it / STAGES;
                    if (!mbar_wait(&full[s], r & 1, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t sa = smem_u32(smem + s * L::STAGE);
                    const uint32_t sb = sa + L::A_BYTES;
#pragma unroll
                    for (int k4 = 0; k4 < BK / 16; ++k4)
                        mma_bf16(acc, sw128_desc(sa + k4 * 32), sw128_desc(sb + k4 * 32), idesc,
                                 (kk > 0 || k4 > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[b]);
            }
            if (!ok) {
                // let the MMAs already issued drain before TMEM is freed
                mma_commit(&tfull[0]);
                mbar_wait(&tfull[0], 0, abort_flag, true);
            }
        }
    } else {
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        int tl = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
            const int b = tl & 1, u = tl >> 1;
            if (!mbar_wait(&tfull[b], u & 1, abort_flag)) { ok = false; break; }
            fence_after();
            const int pr = tile / ntl, tt = tile - pr * ntl;
            const int m0 = (tt % Mt) * BM, n0 = (tt / Mt) * BN;
            const int row = m0 + 32 * q + lane;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + c), r);
                store_chunk(args.p[pr], row, n0 + c, r);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    if (!ok) {
        *abort_flag = 1;
        for (int pr = 0; pr < args.nprob; ++pr)
            if (args.p[pr].flags) atomicOr(args.p[pr].flags, FLAG_TIMEOUT);
    }
    __syncwarp();
    // after a failure anywhere, wait (bounded) for the producer's copies in flight
    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int it = issued > STAGES ? issued - STAGES : 0; it < issued; ++it)
            mbar_wait(&full[it % STAGES], (it / STAGES) & 1, abort_flag, true);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
    }
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared::cluster address of this CTA's variable `p` in cluster CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(const void *p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}

// Arrive on an mbarrier given by its shared::cluster address (this CTA's or the peer's).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}

// TMA load into this CTA's shared memory whose completion is signalled on the
// mbarrier at shared::cluster address `bar`, which may be the peer CTA's
// (.cta_group::2: the barrier sits in either CTA of the pair).
__device__ __forceinline__ void tma_load_3d_pair(void *smem_dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                                 int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 "
        "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier at shared::cluster address `bar` once every MMA this
// thread issued so far has completed (on both CTAs of the pair).
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Two-SM kernel (tcgen05 cta_group::2): a cluster of two CTAs computes one
// 256 x BN output tile with M = 256 MMAs issued by the even CTA.  Each CTA
// TMA-loads, into its own shared memory, its 128 rows of the A tile and its
// BN/2 rows of the B tile (both bf16 split planes of one k block per stage),
// so per SM the operand traffic per flop is half that of a one-CTA 128 x BN
// tile and the same shared memory holds twice the k depth of look-ahead.
// Each CTA's tensor memory holds the accumulator rows of its own 128 output
// rows over all BN columns, and each CTA's epilogue stores them.
//   full[s]   (even CTA): both CTAs' loads of stage s landed (tx bytes of both);
//   empty[s]  (each CTA): the MMAs reading stage s finished (commit to both);
//   tfull[b]  (each CTA): accumulator b is complete (commit to both);
//   tempty[b] (even CTA): both CTAs' epilogues have drained accumulator b.
// Planes: the three retained products x0 y0, x0 y1, x1 y0 are issued from
// one stage, so every plane tile is loaded once per k block.
template <int BN, int STAGES>
struct PairLayout {
    static constexpr int BNH = BN / 2;
    static constexpr int A_PLANE = BM * BK * 2;
    static constexpr int B_PLANE = BNH * BK * 2;
    static constexpr int STAGE = 2 * (A_PLANE + B_PLANE);
    static constexpr int BAR = STAGES * STAGE;
    static constexpr int TOTAL = BAR + (2 * STAGES + 4) * 8 + 16 + 1024;
    static_assert(B_PLANE % 1024 == 0, "B tile rows must fill whole 128-byte swizzle atoms");
    static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "MMA N for M = 256");
};

constexpr int PAIR_TMEM_COLS = 512;

template <int BN, int STAGES, int P>
__global__ void __launch_bounds__(192, 1) k_tc_gemm_pair(const __grid_constant__ TcArgs<P> args) {
    using L = PairLayout<BN, STAGES>;
    const TcParams &p = args.p[0];  // shape: the same for every problem
    constexpr int BNH = L::BNH;
    extern __shared__ uint8_t smem_raw[];
    // same offset in both CTAs: the MMA addresses both CTAs' tiles with one descriptor
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + L::BAR);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;  // [2]
    uint64_t *tempty = tfull + 2;      // [2]
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool lead = (rank == 0);
    const int Mt2 = (p.M + 2 * BM - 1) / (2 * BM), Nt = (p.N + BN - 1) / BN;
    const int ntl = Mt2 * Nt, ntiles = ntl * args.nprob;  // tiles of problem pr: [pr ntl, (pr + 1) ntl)
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    const int total = p.kblocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);  // 4 epilogue warps in each CTA
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {  // one warp of each CTA allocates the pair's tensor memory together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(PAIR_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    cluster_sync();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    int issued = 0;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            for (int t = cid; t < ntiles && ok; t += ncl) {
                const int pr = t / ntl, tt = t - pr * ntl;
                const int m0 = (tt % Mt2) * 2 * BM + (int)rank * BM, n0 = (tt / Mt2) * BN + (int)rank * BNH;
                const CUtensorMap *tmA = &args.a[pr], *tmB = &args.b[pr];
                for (int kk = 0; kk < total; ++kk, ++it) {
                    const int s = it % STAGES, r = it / STAGES;
                    if (!mbar_wait(&empty[s], (r & 1) ^ 1, abort_flag)) { ok = false; break; }
                    const uint32_t fb = lead ? smem_u32(&full[s]) : peer_addr(&full[s], 0);
                    if (lead) mbar_expect_tx(&full[s], 2 * L::STAGE);
                    uint8_t *sa = smem + s * L::STAGE;
                    uint8_t *sb = sa + 2 * L::A_PLANE;
                    // [A plane 0 | A plane 1 | B plane 0 | B plane 1]
                    tma_load_3d_pair(sa, tmA, fb, kk * BK, m0, 0);
                    tma_load_3d_pair(sa + L::A_PLANE, tmA, fb, kk * BK, m0, 1);
                    tma_load_3d_pair(sb, tmB, fb, kk * BK, n0, 0);
                    tma_load_3d_pair(sb + L::B_PLANE, tmB, fb, kk * BK, n0, 1);
                    issued = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lead && lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)((2 * BM) >> 4) << 24);
            int it = 0, tl = 0;
            for (int t = cid; t < ntiles && ok; t += ncl, ++tl) {
                const int b = tl & 1, u = tl >> 1;
                if (!mbar_wait(&tempty[b], (u & 1) ^ 1, abort_flag)) { ok = false; break; }
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * BN);
                for (int kk = 0; kk < total; ++kk, ++it) {
                    const int s = it % STAGES, r = it / STAGES;
                    if (!mbar_wait(&full[s], r & 1, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t sa0 = smem_u32(smem + s * L::STAGE), sa1 = sa0 + L::A_PLANE;
                    const uint32_t sb0 = sa0 + 2 * L::A_PLANE, sb1 = sb0 + L::B_PLANE;
#pragma unroll
                    for (int k4 = 0; k4 < BK / 16; ++k4)
                        mma_bf16_pair(acc, sw128_desc(sa0 + k4 * 32), sw128_desc(sb0 + k4 * 32), idesc,
                                      (kk > 0 || k4 > 0) ? 1u : 0u);
#pragma unroll
                    for (int k4 = 0; k4 < BK / 16; ++k4)
                        mma_bf16_pair(acc, sw128_desc(sa0 + k4 * 32), sw128_desc(sb1 + k4 * 32), idesc, 1u);
#pragma unroll
                    for (int k4 = 0; k4 < BK / 16; ++k4)
                        mma_bf16_pair(acc, sw128_desc(sa1 + k4 * 32), sw128_desc(sb0 + k4 * 32), idesc, 1u);
                    mma_commit_pair(smem_u32(&empty[s]));
                    mma_commit_pair(peer_addr(&empty[s], 1));
                }
                if (!ok) break;
                mma_commit_pair(smem_u32(&tfull[b]));
                mma_commit_pair(peer_addr(&tfull[b], 1));
            }
            if (!ok) {
                // let the MMAs already issued drain before the tensor memory is freed
                mma_commit_pair(smem_u32(&tfull[0]));
                mbar_wait(&tfull[0], 0, abort_flag, true);
            }
        }
    } else {
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        int tl = 0;
        for (int t = cid; t < ntiles; t += ncl, ++tl) {
            const int b = tl & 1, u = tl >> 1;
            if (!mbar_wait(&tfull[b], u & 1, abort_flag)) { ok = false; break; }
            fence_after();
            const int pr = t / ntl, tt = t - pr * ntl;
            const int m0 = (tt % Mt2) * 2 * BM + (int)rank * BM, n0 = (tt / Mt2) * BN;
            const int row = m0 + 32 * q + lane;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + c), r);
                store_chunk(args.p[pr], row, n0 + c, r);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(lead ? smem_u32(&tempty[b]) : peer_addr(&tempty[b], 0));
        }
    }
    if (!ok) {
        *abort_flag = 1;
        for (int pr = 0; pr < args.nprob; ++pr)
            if (args.p[pr].flags) atomicOr(args.p[pr].flags, FLAG_TIMEOUT);
    }
    __syncwarp();
    // after a failure, the even CTA waits (bounded) for the copies in flight of both CTAs
    if (lead && warp == 0 && lane == 0 && *abort_flag) {
        for (int it = issued > STAGES ? issued - STAGES : 0; it < issued; ++it)
            mbar_wait(&full[it % STAGES], (it / STAGES) & 1, abort_flag, true);
    }
    fence_before();
    cluster_sync();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PAIR_TMEM_COLS)
                     : "memory");
    }
    cluster_sync();
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool ensure_encode() {
    if (g_encode) return true;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return true;
}

bool make_map(CUtensorMap *m, const PackView &v, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)v.kp, (cuuint64_t)v.rows, (cuuint64_t)v.planes};
    cuuint64_t strides[2] = {(cuuint64_t)v.kp * 2, (cuuint64_t)v.plane_pitch * 2};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)v.base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int STAGES>
void set_attr() {
    cudaFuncSetAttribute(k_tc_gemm<BN, STAGES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Layout<BN, STAGES>::TOTAL);
    cudaFuncSetAttribute(k_tc_gemm<BN, STAGES, TC_MAX_BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Layout<BN, STAGES>::TOTAL);
}

}  // namespace

// Segment lists: (a plane, b plane) per retained product of split planes.
uint32_t tc_seg_pairs(int nsplit, int *nseg) {
    if (nsplit == 1) { *nseg = 1; return 0u; }
    if (nsplit == 2) {
        *nseg = 3;  // x0y0, x0y1, x1y0
        return (0u << 0) | ((0u << 2 | 1u) << 4) | ((1u << 2 | 0u) << 8);
    }
    *nseg = 6;  // + x0y2, x1y1, x2y0
    return (0u) | ((0u << 2 | 1u) << 4) | ((1u << 2 | 0u) << 8) | ((0u << 2 | 2u) << 12) | ((1u << 2 | 1u) << 16) |
           ((2u << 2 | 0u) << 20);
}

void tc_init_attrs() {
    set_attr<256, 4>();
    set_attr<128, 6>();
    cudaFuncSetAttribute(k_tc_gemm_pair<256, 3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PairLayout<256, 3>::TOTAL);
    cudaFuncSetAttribute(k_tc_gemm_pair<192, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PairLayout<192, 4>::TOTAL);
    cudaFuncSetAttribute(k_tc_gemm_pair<256, 3, TC_MAX_BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PairLayout<256, 3>::TOTAL);
    cudaFuncSetAttribute(k_tc_gemm_pair<192, 4, TC_MAX_BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PairLayout<192, 4>::TOTAL);
}

// Two-SM pair kernel for wide two-plane products (APF_GEMM_PAIR=0: one-CTA tiles only).
static bool pair_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("APF_GEMM_PAIR");  // tuning knob; default on
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

int tc_init() { return ensure_encode() ? APF_OK : APF_ECUDA; }

// How many two-CTA clusters of the pair kernel can be resident at once (the
// SMs of a pair must share a GPC, so this can be below half the SM count).
static int max_pair_clusters() {
    static int v = -1;
    if (v < 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(192);
        cfg.dynamicSmemBytes = PairLayout<256, 3>::TOTAL;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_tc_gemm_pair<256, 3, 1>, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 1 << 20;  // unknown: bounded by the SM count below
        }
        v = n;
    }
    return v;
}

namespace {

template <int P, typename K>
cudaError_t launch_args(apf_ctx *c, K kern, bool pair, unsigned grid, int smem, cudaStream_t s, const TcArgs<P> &args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (pair) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = 2;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args);
    if (e == cudaSuccess) c->launches++;
    return e;
}

// Fill the tensor maps and parameters of nprob problems and launch kernel
// variant `kind` (0: one-CTA 128-wide, 1: one-CTA 256-wide, 2: pair 256, 3: pair 192).
template <int P>
int launch_variant(apf_ctx *c, int kind, int nprob, const TcProblem *pb, const TcParams &base, unsigned grid,
                   cudaStream_t s) {
    TcArgs<P> args;
    memset(&args, 0, sizeof args);
    args.nprob = nprob;
    const int brows = kind == 0 ? 128 : kind == 1 ? 256 : kind == 2 ? 128 : 96;
    for (int i = 0; i < nprob; ++i) {
        if (!make_map(&args.a[i], pb[i].A, BM) || !make_map(&args.b[i], pb[i].B, brows))
            return set_err(c, APF_ECUDA, "tensor map encode failed (M=%d N=%d kp=%lld)", base.M, base.N, pb[i].A.kp);
        TcParams q = base;
        q.out_re = pb[i].out_re; q.out_im = pb[i].out_im;
        q.in_re = pb[i].in_re ? pb[i].in_re : pb[i].out_re;
        q.in_im = pb[i].in_im ? pb[i].in_im : pb[i].out_im;
        q.flags = pb[i].flags;
        args.p[i] = q;
    }
    cudaError_t e = cudaSuccess;
    switch (kind) {
        case 0: e = launch_args(c, k_tc_gemm<128, 6, P>, false, grid, Layout<128, 6>::TOTAL, s, args); break;
        case 1: e = launch_args(c, k_tc_gemm<256, 4, P>, false, grid, Layout<256, 4>::TOTAL, s, args); break;
        case 2: e = launch_args(c, k_tc_gemm_pair<256, 3, P>, true, grid, PairLayout<256, 3>::TOTAL, s, args); break;
        default: e = launch_args(c, k_tc_gemm_pair<192, 4, P>, true, grid, PairLayout<192, 4>::TOTAL, s, args); break;
    }
    if (e != cudaSuccess) return check_cuda(c, e, "tensor-core GEMM launch");
    return APF_OK;
}

}  // namespace

int tc_gemm_n(apf_ctx *c, int nprob, const TcProblem *pb, int nsplit, int M, int N, int n_cplx, float alpha,
              float beta, long long ldo, long long ldi, cudaStream_t s) {
    if (M <= 0 || N <= 0 || nprob <= 0) return APF_OK;
    if (nprob > TC_MAX_BATCH) return set_err(c, APF_EINVAL, "tc_gemm_n: %d problems > %d", nprob, TC_MAX_BATCH);
    if (!ensure_encode()) return set_err(c, APF_ECUDA, "cuTensorMapEncodeTiled unavailable");
    for (int i = 0; i < nprob; ++i)
        if (pb[i].A.kp != pb[i].B.kp || pb[i].A.kp % BK != 0 || pb[i].A.kp != pb[0].A.kp)
            return set_err(c, APF_EINVAL, "tc_gemm: K mismatch (%lld vs %lld)", pb[i].A.kp, pb[i].B.kp);
    const long long kp = pb[0].A.kp;
    TcParams p{};
    p.M = M; p.N = N; p.n_cplx = n_cplx;
    p.kblocks = (int)(kp / BK);
    p.seg_pairs = tc_seg_pairs(nsplit, &p.nseg);
    p.alpha = alpha; p.beta = beta;
    p.ldo = ldo;
    p.ldi = pb[0].in_re ? ldi : ldo;
    // Tile width: score the wave utilisation of 256- and 128-wide tiles.
    static int num_sms = 0;
    if (!num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (num_sms <= 0) num_sms = 148;
    }
    auto util = [&](int bn) {
        long long t = (long long)nprob * ((N + bn - 1) / bn) * ((M + BM - 1) / BM);
        long long waves = (t + num_sms - 1) / num_sms;
        return (double)t / (double)(waves * num_sms);
    };
    // 128 x 256 tiles need ~25% less L2->SM operand traffic per flop; take them
    // unless they waste much more of the last wave
    bool wide = (N > 128) && util(256) >= 0.7 * util(128);
    int bn = wide ? 256 : 128;
    long long ntiles = (long long)nprob * ((N + bn - 1) / bn) * ((M + BM - 1) / BM);
    // SMs left free for kernels of other streams: none by default, since the
    // library runs one solve at a time per GPU and a stream's kernels follow
    // each other (a caller that overlaps its own kernels may reserve some)
    static int reserve = -1;
    if (reserve < 0) {
        const char *e = getenv("APF_GEMM_RESERVED_SMS");  // tuning knob; default 0
        reserve = e ? atoi(e) : 0;
        if (reserve < 0 || reserve > num_sms / 2) reserve = 0;
        if (num_sms <= 64) reserve = 0;
    }
    unsigned grid = (unsigned)std::min<long long>(ntiles, num_sms - reserve);
    int kind = wide ? 1 : 0;
    const int mt = (M + BM - 1) / BM;
    // Pair tiles (256 x BN over two SMs) for wide two-plane products; the tile
    // width BN in {256, 192} that fills the waves of pair slots best.
    const int pair_slots = std::max(1, std::min(max_pair_clusters(), (num_sms - reserve) / 2));
    if (pair_enabled() && nsplit == 2 && mt >= 2 && N >= 256) {
        auto pair_util = [&](int pbn) {
            long long t = (long long)nprob * ((M + 2 * BM - 1) / (2 * BM)) * ((N + pbn - 1) / pbn);
            long long waves = (t + pair_slots - 1) / pair_slots;
            return (double)t / (double)(waves * pair_slots);
        };
        const int pbn = pair_util(192) > 1.1 * pair_util(256) ? 192 : 256;
        kind = pbn == 256 ? 2 : 3;
        long long ntp = (long long)nprob * ((M + 2 * BM - 1) / (2 * BM)) * ((N + pbn - 1) / pbn);
        grid = (unsigned)(2 * std::min<long long>(ntp, pair_slots));
    }
    int pi = -1;
    if (c->prof_on && 2 * (c->prof_used + 1) <= (int)c->prof_ev.size()) {
        pi = c->prof_used++;
        // complex m x k x n product: M = m, N = 2n, kp ~ 2k real
        double alg = 2.0 * (double)M * (double)N * (double)kp * nprob;
        c->prof_alg[pi] = alg;
        c->prof_hw[pi] = alg * p.nseg;
        record_event(c, c->prof_ev[2 * pi], s);
    }
    int rc = nprob == 1 ? launch_variant<1>(c, kind, 1, pb, p, grid, s)
                        : launch_variant<TC_MAX_BATCH>(c, kind, nprob, pb, p, grid, s);
    if (rc != APF_OK) return rc;
    if (pi >= 0) record_event(c, c->prof_ev[2 * pi + 1], s);
    return APF_OK;
}

int tc_gemm(apf_ctx *c, const PackView &A, const PackView &B, int nsplit, int M, int N, int n_cplx, float alpha,
            float beta, float *out_re, float *out_im, long long ldo, const float *in_re, const float *in_im,
            long long ldi, cudaStream_t s) {
    TcProblem pb{A, B, out_re, out_im, in_re, in_im, c->d_flags};
    return tc_gemm_n(c, 1, &pb, nsplit, M, N, n_cplx, alpha, beta, ldo, ldi, s);
}
