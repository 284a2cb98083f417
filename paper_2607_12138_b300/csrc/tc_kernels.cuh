// H1 block kernel with the local multiply on the 5th-generation tensor cores (tcgen05).
//
// Same block structure as k_block (apply_kernels.cuh): table packet staged by bulk async
// copies, x staged in shared memory, exact fixed-point in-block dof sums, partials of boundary
// dofs added up by the combine pass.  The difference is stage 2: for an affine H1 cell the local operator is
// c_K * A_ref with one reference matrix shared by all cells (A_ref = M_ref or M_ref^{-1},
// Eq. piola_mass_pullbacks), so a block's local products form one GEMM
//      Z[cells x n] = Xt[cells x k] * A_ref^T,
// issued by one thread as tcgen05.mma (kind::tf32, M = 128 cells per tile, N = n_loc
// rounded up to 16, K = n_loc rounded up to 8):
//   * each thread writes its cell's signed local vector (row of Xt) straight into tensor
//     memory with tcgen05.st -- row = TMEM lane, k = column -- split into a TF32 "big" part
//     and the exact FP32 remainder ("small");
//   * A_ref, pre-split the same way and pre-arranged in the canonical no-swizzle K-major
//     core-matrix layout (8 rows x 16 bytes per core matrix) at setup, arrives in shared
//     memory with one bulk copy;
//   * Z = Xbig*Abig + Xbig*Asmall + Xsmall*Abig accumulates in FP32 in tensor memory
//     (the 3xTF32 split: about FP32 accuracy), completion signalled by tcgen05.commit on an
//     mbarrier;
//   * each thread reads its row back with tcgen05.ld and continues as in k_block.
// Tensor memory: 128 columns per 128-cell tile ([Xbig | Xsmall | Z]), one or two tiles, allocated
// and released by warp 0; every wait is bounded and every exit path releases it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "apply_kernels.cuh"

namespace bras {

template <int NLOC> struct TcShape {
    static constexpr int K = (NLOC + 7) / 8 * 8;     // reduction dim, multiple of 8 (tf32 K step)
    static constexpr int N = (NLOC + 15) / 16 * 16;  // output dim, multiple of 16 (M = 128)
    static constexpr int TILE_COLS = 128;            // per-tile TMEM columns: Xbig | Xsmall | Z
    static_assert(2 * K + N <= TILE_COLS, "tile does not fit 128 TMEM columns");
    static constexpr uint32_t B_BYTES = (uint32_t)N * K * 4;   // one split of A_ref
};

// Byte offset of element (row n, col k) of an N x K K-major operand in the no-swizzle
// canonical layout: core matrix (n/8, k/4) at ((n/8) * (K/4) + k/4) * 128 bytes, row n%8 at
// 16 bytes each, element k%4 at 4 bytes each.  Leading (K) core-matrix stride 128 bytes,
// stride (N) core-matrix-group stride (K/4) * 128 bytes.
__host__ __device__ inline uint32_t umma_kmajor_offset(int n, int k, int K) {
    return (uint32_t)(((n / 8) * (K / 4) + k / 4) * 128 + (n % 8) * 16 + (k % 4) * 4);
}

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
    // base offset 0, absolute-offset mode off, swizzle mode 0 (none)
    return d;
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128.
template <int N> __device__ __forceinline__ uint32_t umma_idesc_tf32_m128() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
        "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Ties registers written by tcgen05.ld to a point after tcgen05.wait::ld, so that no use of
// them is scheduled before the wait.
template <int N> __device__ __forceinline__ void reg_fence(uint32_t (&v)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) asm volatile("" : "+r"(v[j]));
}

// D[tmem] (+)= A[tmem] * B[smem desc]^T, kind::tf32, one thread.
__device__ __forceinline__ void umma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// Bytes reserved for the B tiles, a multiple of 128 (one right-hand side: the scan scratch of
// stage 3 takes the region over once the GEMM is done).
template <int NLOC>
__host__ __device__ constexpr uint32_t tc_btile_region() {
    return (2 * TcShape<NLOC>::B_BYTES + 127u) & ~127u;
}

struct TcArgs {
    BlockArgs A;
    const unsigned char* btile;   // [Abig | Asmall] pre-arranged, 2 * N * K * 4 bytes
};

// MR = false: one cell per TMEM lane, one right-hand side per CTA (as k_block).  TPC = 1: one
// thread per cell, blockDim / 128 tiles.  TPC = 2: two threads per cell, 256 threads per
// 128-cell tile; in each group of eight warps, warps 0-3 take the even and warps 4-7 the odd
// 8-column groups of the tile's tensor-memory rows (64 registers a thread: four 256-thread or
// two 512-thread CTAs share an SM).
// MR = true (TPC = 1): one CTA per cell block walks the right-hand sides in chunks of 4; the
// block's ne * 4 items (cell, rhs) fill the tensor-memory lanes in passes of blockDim items
// (two 128-lane tiles), each pass one GEMM (the E*R rows of the local product on the M side).
// Stage 3 adds every product to its dof's 64-bit fixed-point accumulator (apply_kernels.cuh);
// with one right-hand side the accumulators take the staged vector's bytes over (dead once the
// local vectors are in tensor memory) and are cleared while the GEMM runs.
template <int NLOC, int OP, bool MR = false, int TPC = 1>
__global__ void __launch_bounds__(TPC == 2 ? 512 : 256, TPC == 2 ? 2 : (MR ? 1 : 2))
k_block_tc(const TcArgs TA, const float* __restrict__ x, float* __restrict__ y, float* __restrict__ part, int nrhs,
           int vec_ok) {
    static_assert(TPC == 1 || (TPC == 2 && !MR), "two threads per cell only for one right-hand side a CTA");
    using Sh = TcShape<NLOC>;
    constexpr int K = Sh::K, N = Sh::N;
    constexpr int CW = MR ? Chunk<float>::CW : 1;
    const int lanes = blockDim.x / TPC;                       // items (TMEM lanes) per pass
    const int tiles = lanes / 128;                            // 128 lanes per tile
    const uint32_t TMEM_COLS = (uint32_t)tiles * Sh::TILE_COLS;   // 128 or 256
    const BlockArgs& A = TA.A;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);   // [0] tab A, [1] tab B, [2] B tile, [3] MMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + 64);
    int* fx = reinterpret_cast<int*>(smem_raw + 80);             // [0, 1] ex per chunk parity, [2] ec
    unsigned char* btile = smem_raw + 128;                       // 2 * B_BYTES, 128-B aligned
    unsigned char* tab = btile + tc_btile_region<NLOC>();
    float* xs = reinterpret_cast<float*>(tab + ((A.max_pkt + 127u) & ~127u));   // [u][CW] staged x
    // [u][CW] accumulators: over the staged vector (one right-hand side), after it (MR)
    long long* ys = MR ? reinterpret_cast<long long*>(xs + ((A.max_u * CW + 3) & ~3)) : reinterpret_cast<long long*>(xs);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int lt = TPC == 2 ? (warp >> 3) * 128 + (tid & 127) : tid;   // this thread's lane in the pass
    const int half = TPC == 2 ? ((warp >> 2) & 1) : 0;                  // its column groups (TPC = 2)
    // one work item per CTA: a block (MR), or a (block, rhs) pair
    const int b = MR ? blockIdx.x : blockIdx.x / nrhs;
    const int e0 = A.blk_e0[b], ne = A.blk_e0[b + 1] - e0;
    const int u0 = A.blk_u0[b], nu = A.blk_u0[b + 1] - u0;
    const int nint = A.blk_nint[b];
    const uint32_t sa = pkt_size_a(nu, false), sb = pkt_size_b((uint32_t)(ne * NLOC), false);
    pdl_launch();
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        mbar_fence_init();
        const unsigned char* src = A.pkt + A.blk_pkt[b];
        mbar_expect_tx(&bars[0], sa);
        bulk_copy_g2s(tab, src, sa, &bars[0]);
        mbar_expect_tx(&bars[1], sb);
        bulk_copy_g2s(tab + sa, src + sa, sb, &bars[1]);
        mbar_expect_tx(&bars[2], 2 * Sh::B_BYTES);
        bulk_copy_g2s(btile, TA.btile, 2 * Sh::B_BYTES, &bars[2]);
        fx[0] = fx[1] = fx[2] = kExpZero;
    }
    if (warp == 0) tmem_alloc(tmem_slot, TMEM_COLS);
    pdl_wait();   // x, the cell factors, y and the partials belong to the stream's order from here
    const float cfac = lt < ne ? static_cast<const float*>(A.scale)[e0 + lt] : 0.f;   // this thread's cell factor
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (lt < ne && (TPC == 1 || half == 0)) atomicMax(&fx[2], exp_bound(cfac));
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t tile_col = (uint32_t)(TPC == 2 ? (warp >> 3) : (warp >> 2)) * Sh::TILE_COLS;
    const int32_t* ids = reinterpret_cast<const int32_t*>(tab);
    const uint16_t* dmul = reinterpret_cast<const uint16_t*>(tab + pkt_off_d(nu));
    const uint16_t* loc = reinterpret_cast<const uint16_t*>(tab + sa);

    bool ok = cta_wait(&bars[0], 0, A.status, true);
    bool tmem_live = true;   // block-uniform
    int pending = -1;        // (thread 0) parity of a committed GEMM whose completion was not seen
    uint32_t commits = 0;    // GEMMs committed on bars[3] so far (its phase parity)
    const int nchunk = MR ? (nrhs + CW - 1) / CW : 1;
    for (int ch = 0; ch < nchunk && ok; ++ch) {
        const int r0 = MR ? ch * CW : blockIdx.x % nrhs;
        const int rc = MR ? min(CW, nrhs - r0) : 1;
        const bool vec = MR && vec_ok && rc == CW;
        const int64_t p0 = MR ? (int64_t)A.blk_p0[b] : (int64_t)r0 * A.npart + A.blk_p0[b];
        int* fxe = &fx[ch & 1];
        if (tid == 0) fx[(ch + 1) & 1] = kExpZero;   // the next chunk's bound (its readers are done)
        const FxAcc acc{ys, (nu * CW + 1) & ~1, A.fx_lo};
        if constexpr (MR) acc.clear(acc.count);
        uint32_t amax = 0;   // largest |staged value| bits
        if constexpr (MR) {
            using V = Chunk<float>::V;
            for (int u = tid; u < nu; u += 4 * blockDim.x) {
                V v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int uu = u + k * blockDim.x;
                    if (uu < nu) v[k] = ld_seg(x + (size_t)ids[uu] * nrhs + r0, rc, vec);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int uu = u + k * blockDim.x;
                    if (uu < nu) {
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            if (OP == OP_BRAS) vget(v[k], j) = div_by_count(vget(v[k], j), dmul[uu]);
                            amax = max(amax, abs_bits(vget(v[k], j)));
                        }
                        reinterpret_cast<V*>(xs)[uu] = v[k];
                    }
                }
            }
        } else {
            // up to 8 loads in flight per thread and pass (blocks of <= 256 cells stage ~8 dofs a
            // thread: a deeper unroll only adds predicated-off slots)
            for (int u = tid; u < nu; u += 8 * blockDim.x) {
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int uu = u + k * blockDim.x;
                    v[k] = uu < nu ? (x + r0)[dof_offset(ids[uu], nrhs)] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int uu = u + k * blockDim.x;
                    if (uu < nu) {
                        const float w = (OP == OP_BRAS) ? div_by_count(v[k], dmul[uu]) : v[k];
                        amax = max(amax, abs_bits(w));
                        xs[uu] = w;
                    }
                }
            }
        }
        const int emax = exp_bound_bits(amax);
        if (emax > kExpZero) atomicMax(fxe, emax);
        if (ch == 0) {
            ok = cta_wait(&bars[1], 0, A.status, ok);
            if (!ok) break;
        } else {
            __syncthreads();
        }
        // the block's fixed-point scale
        bool bad;
        const int kx = fx_scale<float>(*fxe, fx[2], A.fx_er, A.fx_top, bad);
        const float sc = pow2<float>(kx);

        const int nitem = ne * CW;
        const int npass = (nitem + lanes - 1) / lanes;   // block-uniform (1 without MR)
        for (int pass = 0; pass < npass; ++pass) {
            // stage 2a: this thread's item row -> tensor memory (big TF32 part, exact remainder)
            const int it = pass * lanes + lt;   // item of this thread (tile lt / 128, lane lt % 128)
            const bool valid = it < nitem;
            const int e = valid ? it / CW : 0;
            const int rr = it % CW;
            // (TPC = 2: the column groups of this thread's half, fixed at compile time per branch)
            auto stage2a = [&](auto hc) {
                constexpr int H = decltype(hc)::value;
                float xl[K];
#pragma unroll
                for (int a = 0; a < K; ++a) xl[a] = 0.f;
                if (valid) {
#pragma unroll
                    for (int a = 0; a < NLOC; ++a)
                        if (TPC == 1 || ((a >> 3) & 1) == H) xl[a] = xs[loc[a * ne + e] * CW + rr];
                }
#pragma unroll
                for (int k0 = 0; k0 < K; k0 += 8) {
                    if (TPC == 2 && ((k0 >> 3) & 1) != H) continue;
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        hi[j] = f32_to_tf32(xl[k0 + j]);
                        lo[j] = __float_as_uint(xl[k0 + j] - __uint_as_float(hi[j]));
                    }
                    tmem_st8(tmem + lane_base + tile_col + k0, hi);
                    tmem_st8(tmem + lane_base + tile_col + K + k0, lo);
                }
                tmem_wait_st();
            };
            if (half == 0) stage2a(std::integral_constant<int, 0>{});
            else stage2a(std::integral_constant<int, 1>{});
            tc_fence_before();
            __syncthreads();

            // stage 2b: one thread issues the 3xTF32 GEMM for the pass's tiles and waits for it;
            // with one right-hand side the others clear the accumulators (over the staged x,
            // read by now) meanwhile
            if constexpr (!MR) acc.clear(acc.count);
            bool done = true;
            if (tid == 0) {
                if (ch == 0 && pass == 0) done = mbar_wait_bounded(&bars[2], A.status);
                if (done) {
                    tc_fence_after();
                    const uint32_t bb = smem_addr(btile), bs = bb + Sh::B_BYTES;
                    constexpr uint32_t LBO = 128, SBO = (K / 4) * 128;
                    const uint32_t idesc = umma_idesc_tf32_m128<N>();
                    const int ptiles = min(tiles, (nitem - pass * lanes + 127) / 128);
                    for (int t = 0; t < ptiles; ++t) {
                        const uint32_t base = tmem + (uint32_t)t * Sh::TILE_COLS;
                        const uint32_t d = base + 2 * K;
#pragma unroll
                        for (int s = 0; s < K / 8; ++s) {
                            const uint64_t db = umma_smem_desc(bb + s * 2 * 128, LBO, SBO);
                            const uint64_t ds = umma_smem_desc(bs + s * 2 * 128, LBO, SBO);
                            umma_tf32_ts(d, base + 8 * s, db, idesc, s > 0 ? 1u : 0u);      // big * big
                            umma_tf32_ts(d, base + 8 * s, ds, idesc, 1u);                   // big * small
                            umma_tf32_ts(d, base + K + 8 * s, db, idesc, 1u);               // small * big
                        }
                    }
                    umma_commit(&bars[3]);
                    const uint32_t par = commits & 1u;
                    done = mbar_wait_parity_bounded(&bars[3], par, A.status);
                    if (!done) pending = (int)par;
                } else {
                    atomicOr(A.status, 2);
                }
            }
            ++commits;
            ok = __syncthreads_and(done) != 0;
            tc_fence_after();
            if (!ok) break;

            // stage 2c: read this item's row of Z, scale, and add each product to its dof's
            // fixed-point accumulator
            // the cell factor times the block scale and 2^-L (add_prescaled)
            const float cs = (MR ? (valid ? static_cast<const float*>(A.scale)[e0 + e] : 0.f) : cfac) * sc *
                             acc_lo_scale(acc.lo_bits);
            auto stage2c = [&](auto hc) {
                constexpr int H = decltype(hc)::value;
                constexpr int G = N / 16;
                auto mine = [](int g) { return TPC == 1 || (g & 1) == H; };
                // all of this thread's column groups in flight, one wait
                uint32_t v[G][16];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (mine(g)) tmem_ld16(tmem + lane_base + tile_col + 2 * K + 16 * g, v[g]);
                tmem_wait_ld();
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (mine(g)) reg_fence(v[g]);
                if (valid) {
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (!mine(g)) continue;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int a = 16 * g + j;
                            if (a < NLOC) acc.add_prescaled(loc[a * ne + e] * CW + rr, __uint_as_float(v[g][j]) * cs);
                        }
                    }
                }
            };
            if (half == 0) stage2c(std::integral_constant<int, 0>{});
            else stage2c(std::integral_constant<int, 1>{});
            tc_fence_before();
            __syncthreads();   // every product added; the next pass may overwrite tensor memory
        }
        if (!ok) break;
        if constexpr (!MR) {
            // every product is accumulated: release the tensor memory now, so that the next CTA on
            // this SM can allocate it while this one stores
            if (warp == 0) {
                tc_fence_after();
                tmem_dealloc(tmem, TMEM_COLS);
            }
            tmem_live = false;
        }
        // totals: interior dofs to y, shared ones to their partial slots
        for (int i = tid; i < nu * rc; i += blockDim.x) {
            const int u = i / rc, rr = i - u * rc;
            const float v = bad ? __int_as_float(0x7fc00000) : acc.value_f32(u * CW + rr, kx);
            store_dof<float, OP, MR>(u, v, nint, ids, dmul, y, part, nrhs, r0 + rr, p0);
        }
        if (MR) __syncthreads();   // the accumulators are read before the next chunk clears them
    }
    // a GEMM committed but not seen complete: drain it before the columns are released
    if (pending >= 0 && tid == 0) mbar_wait_parity_bounded(&bars[3], (uint32_t)pending, A.status);
    tc_fence_before();
    __syncthreads();
    if (tmem_live && warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (tid == 0) {
        // leave after the copies that may still be in flight have landed (the B tile's phase
        // has completed already unless no item got that far)
        if (!ok) {
            mbar_wait_bounded(&bars[0], A.status);
            mbar_wait_bounded(&bars[1], A.status);
        }
        mbar_wait_bounded(&bars[2], A.status);
    }
}

// Shared memory of the tensor-core block kernel: B tiles, the packet, the staged x (one
// right-hand side: also the 8-byte accumulators over it), the multi-RHS accumulators.
template <int NLOC>
size_t tc_smem_bytes(const BlockArgs& A, bool mr = false) {
    const size_t cw = mr ? Chunk<float>::CW : 1;
    const size_t xsb = sizeof(float) * (((size_t)A.max_u * cw + 3) & ~(size_t)3);
    const size_t ysb = 8 * (((size_t)A.max_u * cw + 1) & ~(size_t)1);
    return 128 + (size_t)tc_btile_region<NLOC>() + ((A.max_pkt + 127u) & ~127u) + (mr ? xsb + ysb : std::max(xsb, ysb));
}

template <int NLOC, int OP>
cudaError_t launch_block_tc(const TcArgs& TA, const CombineArgs& G, int nblk, const float* x, float* y, float* part,
                            int nrhs, cudaStream_t st) {
    const bool mr = nrhs > 1 && tc_smem_bytes<NLOC>(TA.A, true) <= (size_t)smem_optin_bytes();
    // one right-hand side: blocks of at most 128 cells take two threads per cell (four CTAs per
    // SM), larger ones one thread per cell over two tiles (measured faster at 256 cells)
    const bool two = !mr && TA.A.max_ne <= 128;
    const size_t smem = tc_smem_bytes<NLOC>(TA.A, mr);
    auto kern = mr ? k_block_tc<NLOC, OP, true, 1> : (two ? k_block_tc<NLOC, OP, false, 2> : k_block_tc<NLOC, OP, false, 1>);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err != cudaSuccess) return err;
    // one or two 128-cell tensor tiles (two threads per cell); multi-RHS: two tiles of items
    // per pass
    const int threads = 256;
    dim3 grid(mr ? nblk : nblk * nrhs);
    const int vec = rows_vectorisable<float>(nrhs, x, y, part) ? 1 : 0;
    err = launch_pdl(kern, grid, dim3(threads), smem, st, TA, x, y, part, nrhs, vec);
    count_launch(1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_group_combine<float, OP>(G, part, TA.A.npart, y, nrhs, mr, st);
}

}  // namespace bras
