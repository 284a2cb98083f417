// Block-fused element kernels: signed gather -> local dense multiply -> scatter.
//
// One CUDA thread block per cell block (up to 256 cells, one thread per cell):
//   0. one thread issues two bulk asynchronous copies (TMA, cp.async.bulk) of the block's
//      contiguous table packet into shared memory: part A (dof ids, multiplicities,
//      incidence offsets) and part B (local indices with signs, incidence lists), each
//      completing on its own mbarrier, so no table load sits on a dependent-latency chain;
//   1. stage the block's dofs in shared memory, x_s[u] = x[ids[u]] (times 1/d_u for BRAS:
//      the right factor D^{-1} of Eq. mhatinvbras_def);
//   2. each thread gathers its cell's local vector with the signs of P (the injection P_K of
//      Sec. 2.2) and multiplies by the local matrix in registers:
//        H1 (affine):   z_K = c_K * A_ref x_K, A_ref = M_ref (mass) or M_ref^{-1} (BRAS),
//                       c_K = rho_K |det J_K| or its reciprocal (Eq. piola_mass_pullbacks);
//                       A_ref sits in shared memory with 16-byte rows, read as 16-byte
//                       broadcasts;
//        H(curl)/H(div): z_K = A_K x_K with A_K = M_K or M_K^{-1} streamed per cell as a
//                       packed symmetric matrix in a cell-interleaved layout (coalesced);
//   3. every signed local result is added to its block-local dof's 64-bit fixed-point
//      accumulator in shared memory (the P^T of Eq. M_PMbrP / mhatinvbras_def): integer sums
//      are exact, so the total does not depend on the order in which copies arrive; dofs with
//      all copies in the block are final (times 1/d for BRAS, the left D^{-1}), the others
//      leave a partial sum;
//   4. k_group_combine finishes the shared dofs, grouped by the set of blocks that hold their
//      copies: one thread per (shared dof, right-hand side) adds the dof's partials up in the
//      group's ascending block order (times 1/d for BRAS).
// No floating-point atomics anywhere: results are bit-reproducible.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

#include "packet.h"

namespace bras {

void count_launch(int k);

enum { OP_MASS = 0, OP_BRAS = 1, OP_DIAG = 2 };
enum { KIND_H1 = 0, KIND_PACKED = 1 };

struct BlockArgs {
    const int32_t* blk_e0;     // [nblk + 1] first cell of each block
    const int32_t* blk_u0;     // [nblk + 1] first block-local dof (prefix of nu)
    const int32_t* blk_nint;   // [nblk] interior dofs (all copies inside the block)
    const int32_t* blk_p0;     // [nblk] first partial slot
    const int64_t* blk_pkt;    // [nblk] byte offset of the block's packet
    const unsigned char* pkt;  // packets
    const void* refmat;        // T[nloc*nloc]   (H1)
    const void* scale;         // T[E]           (H1)
    const void* pk;            // S[npk][Epad]   (packed)
    int* status;               // device status word (bit 0: a bulk-copy wait timed out)
    int64_t Epad;
    int64_t npart;
    int max_u;
    int max_ne;
    uint32_t max_pkt;          // largest packet (bytes)
    // fixed-point dof sums (stage 3): the bound of a block's products is placed at 2^fx_top;
    // each product's integer splits at bit fx_lo into two parts accumulated in two 32-bit
    // words that cannot overflow for the copies one dof has in a block (fx_lo = 0: one 64-bit
    // word); fx_er bounds the row abs-sums of the local operator: < 2^fx_er (H1: of A_ref;
    // vector spaces: of every A_K)
    int fx_top;
    int fx_lo;
    int fx_er;
    // many right-hand sides, streamed cell matrices (k_cell_mr + k_dof_gather): the cells'
    // local-to-global maps in internal cell order (bit 31 = sign of P), each copy's slot in
    // dof-sorted order (copies of a dof by ascending (cell, local index)), the first slot of
    // each dof, 1/d per dof; null when the context was built for fewer right-hand sides
    const int32_t* mr_l2g;     // [E][nloc]
    const int32_t* mr_slot;    // [E][nloc]
    const int64_t* mr_off;     // [n + 1]
    const void* dinv;          // T[n]
    int64_t n_dof;
    int64_t n_cell;
    // float-float copy of the FP64 cell matrices (hi, lo per entry, FP64 layout): set for the
    // float-float mass apply (BRAS_FP64X) of a many-right-hand-side context, else null
    const float2* pk_df;
};

// Shared dofs for the combine pass (tables.cpp), in group order: item j = (global dof, group g)
// with multiplicity sh_d[j]; group g = (first item, block count, first slot entry): the
// partials of its i-th dof sit at grp_slots[first slot entry + k] + i for its k-th block
// (ascending block order).
struct CombineArgs {
    int64_t nsh;
    const int2* items;
    const uint16_t* sh_d;
    const int4* grp;
    const int32_t* grp_slots;
};

// 16-byte groups of a cell's packed matrix (layout: pk_index in packet.h)
template <typename S> struct PkVec;
template <> struct PkVec<float> { static constexpr int G = 4; using V = float4; };
template <> struct PkVec<double> { static constexpr int G = 2; using V = double2; };
template <> struct PkVec<__nv_bfloat16> { static constexpr int G = 8; using V = uint4; };

__device__ __forceinline__ float4 ld_vec(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_vec(const double2* p) { return __ldg(p); }
__device__ __forceinline__ uint4 ld_vec(const uint4* p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ T vec_elem(const float4& v, int j) {
    return (T)(j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w);
}
template <typename T> __device__ __forceinline__ T vec_elem(const double2& v, int j) { return (T)(j == 0 ? v.x : v.y); }
template <typename T> __device__ __forceinline__ T vec_elem(const uint4& v, int j) {   // 8 bfloat16
    const uint32_t w = j < 2 ? v.x : j < 4 ? v.y : j < 6 ? v.z : v.w;
    return (T)__uint_as_float((j & 1) ? (w & 0xFFFF0000u) : (w << 16));
}

// Visit the packed entries (a, q <= a) of this thread's cell in order, 16 bytes per load;
// f(a, q, m) is inlined with compile-time a, q after unrolling.  Layout pk_index (packet.h):
// the groups of a cell sit 32 groups apart inside its tile of 32 cells, so a warp of 32
// consecutive cells reads its tile as one contiguous stream of 512-byte rows.
template <int NLOC, typename T, typename S, typename F>
__device__ __forceinline__ void for_packed(const S* pk_base, int64_t cell, F&& f) {
    using V = typename PkVec<S>::V;
    constexpr int G = PkVec<S>::G, NPK = NLOC * (NLOC + 1) / 2, NG = (NPK + G - 1) / G;
    const V* base = reinterpret_cast<const V*>(pk_base) + (((size_t)(cell >> 5) * NG) << 5) + (size_t)(cell & 31);
    int a = 0, q = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const V v = ld_vec(base + ((size_t)g << 5));
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (g * G + j < NPK) {
                f(a, q, vec_elem<T>(v, j));
                if (++q > a) {
                    ++a;
                    q = 0;
                }
            }
        }
    }
}

// ---- bulk asynchronous copy + mbarrier helpers (sm_90+ PTX) -------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Test the phase of `bar` with the given parity; if it is not complete the thread is suspended
// until it completes or `hint_ns` nanoseconds pass (the suspend-time hint of try_wait), so a
// waiting thread does not spin on the issue slots the other warps of the SM need.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Programmatic dependent launch.  A kernel launched with programmatic stream serialization
// (launch_pdl) may start while its predecessor in the stream is still running: pdl_launch()
// lets the successor start launching once every CTA of this kernel has called it, and
// pdl_wait() blocks until the predecessor has completed with its memory visible.  Kernels call
// pdl_wait() before their first read of data another kernel may write and before their first
// global write; before it they only set up shared memory, barriers and copies of tables that
// never change after setup.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bounded wait on the phase of `bar` with the given parity (barriers reused across phases):
// each try_wait suspends the thread for up to 20 us or until the phase completes; the wait
// gives up after 0.5 s of the global timer (or 2^20 tries), records the failure in `status`
// and tells the caller.
__device__ __forceinline__ bool mbar_wait_parity_bounded(uint64_t* bar, uint32_t parity, int* status) {
    if (mbar_try_wait(bar, parity, 20000u)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 20); ++it) {
        if (mbar_try_wait(bar, parity, 20000u)) return true;
        if (global_ns() - t0 > 500000000ull) break;
    }
    atomicOr(status, 1);
    return false;
}
// Bounded wait on phase 0 of `bar`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, int* status) {
    return mbar_wait_parity_bounded(bar, 0u, status);
}

// v / d for the multiplicity d: FP64 divides; FP32 multiplies by the hardware reciprocal
// approximation of 1/d (one instruction, within one unit in the last place).
__device__ __forceinline__ double div_by_count(double v, uint16_t d) { return v / (double)d; }
__device__ __forceinline__ float rcp_approx(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}
__device__ __forceinline__ float div_by_count(float v, uint16_t d) { return v * rcp_approx((float)d); }

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec4<double> { using type = double2; static constexpr int W = 2; };

template <int N, typename T> struct PadTo {
    static constexpr int W = Vec4<T>::W;
    static constexpr int value = (N + W - 1) / W * W;
};

// Float-float product term: (sh, sl) += (mh + ml) * (vh + vl) to about 2^-48 relative, on the
// FP32 units (B300 runs FP32 at 64x its FP64 rate).  Error-free product of the high parts
// (p + e = mh * vh exactly, by an FMA), first-order cross terms, and a Knuth two-sum into the
// running pair; the _rn intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void df_term(float mh, float ml, float vh, float vl, float& sh, float& sl) {
    const float p = __fmul_rn(mh, vh);
    const float e = __fmaf_rn(mh, vh, -p);
    const float t = __fmaf_rn(mh, vl, __fmaf_rn(ml, vh, e));
    const float s = __fadd_rn(sh, p);
    const float bp = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, t));
}

// (ah, al) += (bh, bl) as float-float pairs (two-sum of the high parts, low parts added).
__device__ __forceinline__ void df_merge(float& ah, float& al, float bh, float bl) {
    const float s = __fadd_rn(ah, bh);
    const float bp = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fsub_rn(bh, bp));
    ah = s;
    al = __fadd_rn(__fadd_rn(al, bl), err);
}

// Streamed FP32/bf16 cell matrices, one right-hand side, n_loc <= 48: ask for two resident
// blocks per SM (at most 128 registers a thread), so that twice as many matrix loads are in
// flight.  Multi-RHS CTAs are shared-memory bound to one per SM and keep each item's local
// vector in registers; n_loc = 70, 84 need the full register file for their accumulators.
template <int KIND, typename T, int NLOC, bool MR = false> struct MinBlocks {
    static constexpr int value = (KIND == KIND_PACKED && sizeof(T) == 4 && !MR && NLOC <= 48) ? 2 : 1;
};

// ---- multi-RHS row segments --------------------------------------------------------------
// A chunk is CW = 16 / sizeof(T) consecutive right-hand sides (4 FP32 or 2 FP64): one 16-byte
// vector per dof row of x, y, the staged x and the staged local results.
template <typename T> struct Chunk {
    using V = typename Vec4<T>::type;   // float4 / double2
    static constexpr int CW = Vec4<T>::W;
};
__device__ __forceinline__ float4 vzero(float4) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ void vadd(float4& a, const float4& b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }
__device__ __forceinline__ void vadd(double2& a, const double2& b) { a.x += b.x; a.y += b.y; }
__device__ __forceinline__ float& vget(float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ double& vget(double2& v, int j) { return j == 0 ? v.x : v.y; }

// Row segment [r0, r0 + rc) of one dof (rc <= CW; the rest of the vector is zero).  vec: rows
// 16-byte aligned and a full chunk.
template <typename T>
__device__ __forceinline__ typename Chunk<T>::V ld_seg(const T* p, int rc, bool vec) {
    using V = typename Chunk<T>::V;
    if (vec) return __ldg(reinterpret_cast<const V*>(p));
    V v = vzero(V{});
#pragma unroll
    for (int j = 0; j < Chunk<T>::CW; ++j)
        if (j < rc) vget(v, j) = p[j];
    return v;
}
template <typename T>
__device__ __forceinline__ void st_seg(T* p, int rc, bool vec, typename Chunk<T>::V v) {
    using V = typename Chunk<T>::V;
    if (vec) {
        *reinterpret_cast<V*>(p) = v;
        return;
    }
#pragma unroll
    for (int j = 0; j < Chunk<T>::CW; ++j)
        if (j < rc) p[j] = vget(v, j);
}

// One thread polls the mbarrier (bounded) while the rest of the CTA sleeps in the CTA barrier;
// returns the block-uniform outcome.  `prior` = false skips the poll and propagates the failure.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, int* status, bool prior) {
    bool ok = true;
    if (threadIdx.x == 0) ok = prior && mbar_wait_parity_bounded(bar, parity, status);
    return __syncthreads_and(ok) != 0;
}

// ---- stage 3: exact fixed-point dof sums -------------------------------------------------
// Every signed local product v of a block is added to its block-local dof's integer
// accumulator as q = rint(v * 2^k) with shared-memory integer atomics.  The integer sums are
// exact, so a dof's total does not depend on the order in which its copies arrive: every apply
// gives the same bits (no floating-point atomics).  The scale comes from an a-priori bound of
// the block's products, |v| < 2^(ex + ec + fx_er) with ex, ec the block's largest exponents of
// the staged x and of the cell factors (H1; 0 for the vector spaces) and fx_er that of the
// local operator's row abs-sums, placed at 2^fx_top: k = fx_top - ex - ec - fx_er.  The total
// is converted back rounded to nearest (FP32: from its two words, FxAcc::value_f32, within
// 2^-38 of the bound besides that rounding); products well below the bound keep an absolute
// resolution of 2^-k = 2^-fx_top of the bound.  With at most 2^h copies of a dof in a block:
//   FP32 and bf16 applies: q = qh 2^L + ql with |ql| <= 2^(L-1), each part summed in a 32-bit
//     word; L = min(22, 30 - h), fx_top = min(L + 21, 31 + L - h) (43 bits for h <= 8, about
//     1e-13 of the bound, far below FP32 rounding).  Both parts come out of FP32 additions
//     with the round-to-integer constant 1.5 * 2^23 (exact for magnitudes below 2^22), so no
//     64-bit float-integer conversion is needed: B300 runs those on its FP64 pipe, at 1/64 of
//     the FP32 rate.
//   FP64 applies: one 64-bit word (fx_lo = 0, fx_top = 61 - h), rounded by the FP64 conversion.
//   The float-float H1 mass apply: q of each half of a product pair split into fx_lo = 31 - h
//     low bits and the rest (fx_top = 60 - 2h, about 2^-48 of the bound for the FP64 result).
constexpr int kExpZero = -100000;   // exponent bound of zero
constexpr int kExpBad = 100000;     // of an infinity or a NaN

// IEEE bits of |v|.  exp_bound_bits is non-decreasing in them (zero, subnormals, normals by
// exponent, infinities, NaNs), so the bound of a set of values is the bound of their largest
// magnitude bits: staging loops keep an unsigned maximum and convert once.
__device__ __forceinline__ uint32_t abs_bits(float v) { return __float_as_uint(v) & 0x7fffffffu; }
__device__ __forceinline__ uint64_t abs_bits(double v) {
    return (uint64_t)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
// E with |v| < 2^E, read off the IEEE exponent field of |v|'s bits
__device__ __forceinline__ int exp_bound_bits(uint32_t bits) {
    if (bits == 0) return kExpZero;
    const int f = (int)(bits >> 23);
    return f == 255 ? kExpBad : (f == 0 ? -126 : f - 126);
}
__device__ __forceinline__ int exp_bound_bits(uint64_t bits) {
    if (bits == 0) return kExpZero;
    const int f = (int)(bits >> 52);
    return f == 2047 ? kExpBad : (f == 0 ? -1022 : f - 1022);
}
__device__ __forceinline__ int exp_bound(float v) { return exp_bound_bits(abs_bits(v)); }
__device__ __forceinline__ int exp_bound(double v) { return exp_bound_bits(abs_bits(v)); }

// Scale exponent k of a block from its exponent bounds; bad = the products are not finite (or
// beyond what the accumulators can hold), and the block then stores NaN.
template <typename T>
__device__ __forceinline__ int fx_scale(int ex, int ec, int er, int top, bool& bad) {
    constexpr int kmin = sizeof(T) == 4 ? -126 : -1022, kmax = sizeof(T) == 4 ? 126 : 1022;
    bad = ex >= kExpBad || ec >= kExpBad;
    if (ex <= kExpZero || ec <= kExpZero) return 0;   // every product is zero
    const int k = top - (ex + ec + er);
    if (k < kmin) bad = true;
    return max(kmin, min(kmax, k));
}

// 2^k as T, k within the normal range of T
template <typename T> __device__ __forceinline__ T pow2(int k);
template <> __device__ __forceinline__ float pow2<float>(int k) { return __int_as_float((k + 127) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ __forceinline__ long long fx_round(float v) { return __float2ll_rn(v); }
__device__ __forceinline__ long long fx_round(double v) { return __double2ll_rn(v); }

// rint(t) for |t| < 2^22 on the FP32 adder: t + 1.5 * 2^23 lands in [2^23, 2^24), where the
// spacing is 1, so the sum is rounded to an integer (ties to even) and its low mantissa bits
// hold that integer plus 2^22.
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;  // its IEEE bits
__device__ __forceinline__ int magic_int(float rounded) { return __float_as_int(rounded) - kRoundMagicBits; }

// Correctly rounded int64 -> float on the integer units (normalise, round to nearest even on
// the dropped bits; a mantissa carry moves into the exponent field by itself).
__device__ __forceinline__ float ll_to_float_rn(long long q) {
    if (q == 0) return 0.f;
    const uint32_t sgn = q < 0 ? 0x80000000u : 0u;
    unsigned long long m = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    const int lz = __clzll((long long)m);
    m <<= lz;                                          // leading one at bit 63
    uint32_t mant = (uint32_t)(m >> 40);               // 24 bits, bit 23 set
    const unsigned long long rest = m << 24;           // the 40 dropped bits, left-aligned
    const unsigned long long half = 0x8000000000000000ull;
    if (rest > half || (rest == half && (mant & 1u))) ++mant;
    return __uint_as_float(sgn | ((uint32_t)(63 - lz + 126) << 23) + mant);
}

// The accumulators of a block: FP32 (lo_bits > 0) two 32-bit words per dof, the low words of
// every dof first and the high words after them (so that the lanes of a warp spread over all
// banks), FP64 (lo_bits = 0) one 64-bit word per dof.  `count` dofs (times right-hand sides).
struct FxAcc {
    long long* base;
    int count;
    int lo_bits;
    // zero the first n 8-byte words (n = count covers both halves, or every 64-bit word)
    __device__ __forceinline__ void clear(int n) const {
        for (int i = threadIdx.x; i < n; i += blockDim.x) base[i] = 0;
    }
    // FP32 product already scaled, s = v 2^k with |s| < 2^(lo_bits + 22), lo_bits <= 22:
    // rint(s) = qh 2^L + ql, qh = rint(s 2^-L) and ql = rint(s - qh 2^L) (the FMA forms that
    // difference exactly; |ql| <= 2^(L-1)), each part by the round-to-integer constant.
    __device__ __forceinline__ void add_scaled(int i, float s) const {
        const float t = __fmul_rn(s, __int_as_float((127 - lo_bits) << 23));
        const float th = __fadd_rn(t, kRoundMagic);
        const float hf = __fsub_rn(th, kRoundMagic);
        const float r = __fmaf_rn(-hf, __int_as_float((127 + lo_bits) << 23), s);
        int* w = reinterpret_cast<int*>(base);
        atomicAdd(w + i, magic_int(__fadd_rn(r, kRoundMagic)));
        atomicAdd(w + count + i, magic_int(th));
    }
    // The same with the product given as t = s 2^-L (the caller folds 2^-L into its scale
    // factor, one multiply less per product): qh = rint(t), t - qh is exact (the fraction of t,
    // or Sterbenz for |t| < 1), and ql = rint((t - qh) 2^L) by one FMA with the round-to-integer
    // constant -- the same two integers as add_scaled(i, t 2^L).  Only where the folded factor
    // falls below FP32's normal range (cell factors 2^40 apart in one block) does it keep fewer
    // bits: those products stay below 2^-29 of the block's bound, and the result is still a
    // fixed function of the inputs.
    __device__ __forceinline__ void add_prescaled(int i, float t) const {
        const float th = __fadd_rn(t, kRoundMagic);
        const float fr = __fsub_rn(t, __fsub_rn(th, kRoundMagic));
        const float tl = __fmaf_rn(fr, __int_as_float((127 + lo_bits) << 23), kRoundMagic);
        int* w = reinterpret_cast<int*>(base);
        atomicAdd(w + i, magic_int(tl));
        atomicAdd(w + count + i, magic_int(th));
    }
    // FP64 product (one 64-bit word, lo_bits = 0)
    __device__ __forceinline__ void add_scaled(int i, double s) const {
        atomicAdd(reinterpret_cast<unsigned long long*>(base) + i, (unsigned long long)fx_round(s));
    }
    __device__ __forceinline__ void add(int i, long long q) const {
        if (lo_bits == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(base) + i, (unsigned long long)q);
            return;
        }
        int* w = reinterpret_cast<int*>(base);
        atomicAdd(w + i, (int)(q & ((1ll << lo_bits) - 1)));
        atomicAdd(w + count + i, (int)(q >> lo_bits));
    }
    __device__ __forceinline__ long long total(int i) const {
        if (lo_bits == 0) return base[i];
        const int* w = reinterpret_cast<const int*>(base);
        return ((long long)w[count + i] << lo_bits) + (long long)w[i];
    }
    // FP32 total times 2^-k from the two words (lo_bits > 0): the high word is exact in FP32
    // (|hi| < 2^22 since totals stay below 2^fx_top <= 2^(L + 21)), the low word is rounded
    // only beyond 2^24 (|lo| <= 2^(L - 1 + h) <= 2^29), and hi 2^L + lo is rounded once by
    // an FMA: within half a unit in the last place plus 2^5 units of 2^-k (below 2^-38 of the
    // block's bound), and a function of the two exact integer sums alone, so every apply still
    // gives the same bits.  Two conversions and an FMA instead of a 64-bit normalisation.
    __device__ __forceinline__ float value_f32(int i, int k) const {
        const int* w = reinterpret_cast<const int*>(base);
        const float hi = __int2float_rn(w[count + i]), lo = __int2float_rn(w[i]);
        return __fmul_rn(__fmaf_rn(hi, __int_as_float((127 + lo_bits) << 23), lo), __int_as_float((127 - k) << 23));
    }
};

// 2^-L for the low-word split at bit L (lo_bits)
__device__ __forceinline__ float acc_lo_scale(int lo_bits) { return __int_as_float((127 - lo_bits) << 23); }

// accumulator -> value: one rounding of the exact integer sum, then the exact power-of-two scale
__device__ __forceinline__ float fx_value(long long q, int k, float) { return ll_to_float_rn(q) * pow2<float>(-k); }
__device__ __forceinline__ double fx_value(long long q, int k, double) { return __ll2double_rn(q) * pow2<double>(-k); }
// accumulator i of a block -> value: FP32 from the two words, FP64 from the 64-bit word
__device__ __forceinline__ float fx_total(const FxAcc& acc, int i, int k, float) { return acc.value_f32(i, k); }
__device__ __forceinline__ double fx_total(const FxAcc& acc, int i, int k, double) {
    return fx_value(acc.total(i), k, 0.0);
}

// Element offset of dof `id` (>= 0) in a [n][nrhs] array: one 32 x 32 -> 64-bit multiply
__device__ __forceinline__ size_t dof_offset(int32_t id, int nrhs) { return (size_t)(uint32_t)id * (uint32_t)nrhs; }

// Stage 3's store of one dof's total: interior dofs to y (times 1/d for BRAS), shared ones to
// their partial slot ([nrhs][npart] from p0; MR: slot-major rows, right-hand side r).
template <typename T, int OP, bool MR>
__device__ __forceinline__ void store_dof(int u, T v, int nint, const int32_t* ids, const uint16_t* dmul,
                                          T* __restrict__ y, T* __restrict__ part, int nrhs, int r, int64_t p0) {
    if (u < nint) (y + r)[dof_offset(ids[u], nrhs)] = (OP == OP_BRAS) ? div_by_count(v, dmul[u]) : v;
    else if (MR) part[(size_t)(p0 + (u - nint)) * nrhs + r] = v;
    else part[p0 + (u - nint)] = v;
}

// Stage 3 of the scatter path (streamed cell matrices): every block-local dof u sums its copies
// zs[incoff[u], incoff[u+1]) in that order (Eq. mhatinvbras_def, the D^{-1} P^T half) and hands
// the total to out(u, v).  A thread takes four dofs at a time so that their shared-memory chains
// overlap; every dof's order is unchanged.
template <typename V, typename Add, typename Out>
__device__ __forceinline__ void dof_run_sums(int nu, const uint16_t* incoff, const V* zs, V zero, Add add, Out out) {
    constexpr int U = 4;
    const int T = blockDim.x;
    for (int u = threadIdx.x; u < nu; u += U * T) {
        int s0[U], cnt[U];
        V acc[U];
        int mx = 0;
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int uu = u + k * T;
            s0[k] = uu < nu ? incoff[uu] : 0;
            cnt[k] = uu < nu ? incoff[uu + 1] - s0[k] : 0;
            acc[k] = zero;
            mx = max(mx, cnt[k]);
        }
        for (int j = 0; j < mx; ++j) {
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (j < cnt[k]) acc[k] = add(acc[k], zs[s0[k] + j]);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int uu = u + k * T;
            if (uu < nu) out(uu, acc[k]);
        }
    }
}

// Stage 4: one thread per (shared dof, rhs); every dof adds its partials in ascending block
// order (0 + p_0 + p_1 + ...) and stores the total to y (times 1/d for BRAS).  Consecutive
// threads take consecutive dofs of a group, so the partial reads coalesce and the group's
// record and slots are shared through L1.  slot_major: partials laid out [npart][nrhs], else
// [nrhs][npart].
template <typename T, int OP>
__global__ void __launch_bounds__(256) k_group_combine(const CombineArgs G, const T* __restrict__ part, int64_t npart,
                                                       T* __restrict__ y, int nrhs, int slot_major) {
    pdl_launch();
    pdl_wait();
    const int64_t total = G.nsh * nrhs;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = nrhs == 1 ? q : q / nrhs;
        const int r = (int)(q - j * nrhs);
        const int2 it = __ldg(G.items + j);
        const int4 gr = __ldg(G.grp + it.y);
        const int i = (int)(j - gr.x), cnt = gr.y;
        const int32_t* sl = G.grp_slots + gr.z;
        T acc = T(0);
        for (int k0 = 0; k0 < cnt; k0 += 4) {
            T v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k0 + k < cnt) {
                    const int64_t slot = (int64_t)__ldg(sl + k0 + k) + i;
                    v[k] = __ldg(part + (slot_major ? slot * nrhs + r : (int64_t)r * npart + slot));
                } else {
                    v[k] = T(0);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k0 + k < cnt) acc += v[k];
        }
        y[(size_t)it.x * nrhs + r] = (OP == OP_BRAS) ? div_by_count(acc, __ldg(G.sh_d + j)) : acc;
    }
}

// Launch with programmatic stream serialization (see pdl_wait): the kernel may begin while its
// predecessor in the stream finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename T, int OP>
cudaError_t launch_group_combine(const CombineArgs& G, const T* part, int64_t npart, T* y, int nrhs, bool slot_major,
                                 cudaStream_t st) {
    if (G.nsh <= 0) return cudaSuccess;
    const int nb = (int)std::min<int64_t>((G.nsh * nrhs + 255) / 256, 148 * 16);
    const cudaError_t err = launch_pdl(k_group_combine<T, OP>, dim3(nb), dim3(256), 0, st, G, part, npart, y, nrhs,
                                       slot_major ? 1 : 0);
    count_launch(1);
    return err != cudaSuccess ? err : cudaGetLastError();
}

__device__ __forceinline__ float4 vsum(float4 a, const float4& b) { vadd(a, b); return a; }
__device__ __forceinline__ double2 vsum(double2 a, const double2& b) { vadd(a, b); return a; }

// Kernel modes.  MR = false: one right-hand side per CTA (grid = blocks x nrhs), vectors read
// with stride nrhs, partial sums laid out [nrhs][npart].  MR = true (multi-RHS): one CTA per
// cell block (grid = blocks) walks the right-hand sides in chunks of CW; each cell of the block
// is CW work items (cell, rhs), rows of x and y move as 16-byte vectors, partial sums are laid
// out [npart][nrhs].  The block's tables (and streamed cell matrices, re-read from L2) serve
// every chunk.
// Stage 3 by kind: H1 blocks add their products into fixed-point accumulators (ys); blocks of
// streamed cell matrices (KIND_PACKED: up to 4 KB of matrix per cell, so the products leave a
// thread in a long stream of loads) write each product to its dof-sorted slot (zs) and sum the
// dofs' runs afterwards, which costs fewer shared-memory operations per copy than the atomics.
template <int NLOC, typename T, typename S, int KIND, int OP, bool MR = false>
__global__ void __launch_bounds__(256, (MinBlocks<KIND, T, NLOC, MR>::value))
k_block(const BlockArgs A, const T* __restrict__ x, T* __restrict__ y, T* __restrict__ part, int nrhs, int vec_ok) {
    constexpr int NPAD = PadTo<NLOC, T>::value;
    constexpr int CW = MR ? Chunk<T>::CW : 1;
    using V = typename Chunk<T>::V;
    constexpr bool FX = KIND == KIND_H1;   // fixed-point accumulators (else dof-sorted scatter)
    // Lagrange (H1) dofs carry no orientation: the sign bit of a local index is only read for
    // H(curl)/H(div)
    constexpr bool SIGNED = KIND == KIND_PACKED;
    constexpr bool XS = KIND == KIND_PACKED && NLOC >= 36 && OP != OP_DIAG;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);             // [0, 1] mbarriers
    int* fx = reinterpret_cast<int*>(smem_raw + 64);                    // [0, 1] ex per chunk parity, [2] ec
    unsigned char* tab = smem_raw + 128;                                 // table packet
    T* xs = reinterpret_cast<T*>(tab + ((A.max_pkt + 127u) & ~127u));  // [u][CW] staged x
    // H1: [u][CW] accumulators; vector spaces: [slot][CW] dof-sorted products (the signed local
    // vectors of n_loc >= 36 wait there first, column e of a [a][cell] array)
    T* after_xs = xs + ((A.max_u * CW + 3) & ~3);
    long long* ys = reinterpret_cast<long long*>(after_xs);
    T* zs = after_xs;
    T* Ms = FX ? reinterpret_cast<T*>(ys + (((size_t)A.max_u * CW + 1) & ~(size_t)1))
               : zs + ((NLOC * A.max_ne * CW + 3) & ~3);                  // [NLOC][NPAD] (H1), 16-B aligned

    const int b = MR ? blockIdx.x : blockIdx.x / nrhs, tid = threadIdx.x;
    const int e0 = A.blk_e0[b], ne = A.blk_e0[b + 1] - e0;
    const int u0 = A.blk_u0[b], nu = A.blk_u0[b + 1] - u0;
    const int nint = A.blk_nint[b];
    const uint32_t m = (uint32_t)(ne * NLOC);
    const uint32_t sa = pkt_size_a(nu, !FX), sb = pkt_size_b(m, !FX);
    pdl_launch();
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        const unsigned char* src = A.pkt + A.blk_pkt[b];
        mbar_expect_tx(&bars[0], sa);
        bulk_copy_g2s(tab, src, sa, &bars[0]);
        mbar_expect_tx(&bars[1], sb);
        bulk_copy_g2s(tab + sa, src + sa, sb, &bars[1]);
        fx[0] = fx[1] = fx[2] = kExpZero;
    }
    if (KIND == KIND_H1) {
        const T* ref = static_cast<const T*>(A.refmat);
        for (int i = tid; i < NLOC * NPAD; i += blockDim.x) {
            const int a = i / NPAD, q = i - a * NPAD;
            const T v = q < NLOC ? ref[a * NLOC + q] : T(0);
            Ms[i] = v;
        }
    }
    pdl_wait();   // x, the cell factors, y and the partials belong to the stream's order from here
    // this thread's cell factor (H1, one cell per thread; multi-RHS items read theirs again)
    const T cfac = (KIND == KIND_H1 && tid < ne) ? static_cast<const T*>(A.scale)[e0 + tid] : T(0);
    __syncthreads();   // barriers and bounds initialised before anyone uses them
    if (FX) {
        int ec = tid < ne ? exp_bound(cfac) : kExpZero;
        for (int e = tid + blockDim.x; e < ne; e += blockDim.x)   // blocks of more cells than threads
            ec = max(ec, exp_bound(static_cast<const T*>(A.scale)[e0 + e]));
        if (ec > kExpZero) atomicMax(&fx[2], ec);
    }
    const int32_t* ids = reinterpret_cast<const int32_t*>(tab);
    const uint16_t* dmul = reinterpret_cast<const uint16_t*>(tab + pkt_off_d(nu));
    const uint16_t* incoff = reinterpret_cast<const uint16_t*>(tab + pkt_off_incoff(nu));
    const uint16_t* loc = reinterpret_cast<const uint16_t*>(tab + sa);
    const uint16_t* pos = reinterpret_cast<const uint16_t*>(tab + sa + pkt_off_pos(m));

    const bool okA = cta_wait(&bars[0], 0, A.status, true);
    const int nchunk = MR ? (nrhs + CW - 1) / CW : 1;
    for (int ch = 0; ch < nchunk; ++ch) {
        const int r0 = MR ? ch * CW : blockIdx.x % nrhs;
        const int rc = MR ? min(CW, nrhs - r0) : 1;
        const bool vec = MR && vec_ok && rc == CW;
        // first partial slot of this block (MR: row of [npart][nrhs])
        const int64_t p0 = MR ? (int64_t)A.blk_p0[b] : (int64_t)r0 * A.npart + A.blk_p0[b];
        int* fxe = &fx[ch & 1];
        const FxAcc acc{ys, (nu * CW + 1) & ~1, A.fx_lo};
        if (FX) {
            if (tid == 0) fx[(ch + 1) & 1] = kExpZero;   // the next chunk's bound (its readers are done)
            acc.clear(acc.count);
        }

        int emax = OP == OP_DIAG ? 1 : kExpZero;   // DIAG: the products are matrix entries (x = 1)
        decltype(abs_bits(T(0))) amax = 0;         // largest |staged value| bits
        if (OP != OP_DIAG && okA) {
            if constexpr (MR) {
                // one 16-byte row segment per dof, four in flight per thread
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
                                if (FX) amax = max(amax, abs_bits(vget(v[k], j)));
                            }
                            reinterpret_cast<V*>(xs)[uu] = v[k];
                        }
                    }
                }
            } else {
                // several loads in flight per thread and pass: 16 for the streamed spaces (many
                // dofs a thread), 4 for H1 (about one to four dofs a thread)
                constexpr int UX = KIND == KIND_H1 ? 4 : 16;
                for (int u = tid; u < nu; u += UX * blockDim.x) {
                    T v[UX];
#pragma unroll
                    for (int k = 0; k < UX; ++k) {
                        const int uu = u + k * blockDim.x;
                        v[k] = uu < nu ? (x + r0)[dof_offset(ids[uu], nrhs)] : T(0);
                    }
#pragma unroll
                    for (int k = 0; k < UX; ++k) {
                        const int uu = u + k * blockDim.x;
                        if (uu < nu) {
                            const T w = (OP == OP_BRAS) ? div_by_count(v[k], dmul[uu]) : v[k];
                            if (FX) amax = max(amax, abs_bits(w));
                            xs[uu] = w;
                        }
                    }
                }
            }
        }
        if (FX && OP != OP_DIAG) emax = exp_bound_bits(amax);
        if (FX && emax > kExpZero) atomicMax(fxe, emax);
        if (ch == 0) {
            if (!cta_wait(&bars[1], 0, A.status, okA)) {   // block-uniform decision
                // let any copy still in flight land before the block's shared memory is released
                if (tid == 0) {
                    mbar_wait_bounded(&bars[0], A.status);
                    mbar_wait_bounded(&bars[1], A.status);
                }
                return;
            }
        } else {
            __syncthreads();
        }
        // H1: the block's fixed-point scale (the bounds and the zeroed accumulators are complete)
        bool bad = false;
        const int kx = FX ? fx_scale<T>(*fxe, fx[2], A.fx_er, A.fx_top, bad) : 0;
        const T sc = pow2<T>(kx);
        const T scl = sc * T(FX && sizeof(T) == 4 ? acc_lo_scale(A.fx_lo) : 1.f);   // FP32: sc 2^-L

        // Work items: (cell e, rhs rr) -> item e * CW + rr.  One item per thread without MR.
        const int nitem = ne * CW;
        if constexpr (XS && !MR) {
            // Large streamed cell matrices (n_loc >= 36): the signed local vector waits in shared
            // memory, column e of a [a][cell] array (only this thread touches it), so that
            // registers hold just the accumulators and the matrix loads in flight; the results go
            // out after a barrier, over the same array.
            const int e = tid;
            T* xt = zs;
            uint64_t neg = 0;
            T zl[NLOC];
#pragma unroll
            for (int a = 0; a < NLOC; ++a) zl[a] = T(0);
            if (e < ne) {
                const uint16_t* L = loc + e;
#pragma unroll
                for (int a = 0; a < NLOC; ++a) {
                    const uint16_t c = L[a * ne];
                    const T v = xs[c & 0x7fff];
                    const bool s = (c & 0x8000) != 0;
                    if (a < 64) neg |= (uint64_t)s << (a & 63);
                    xt[a * ne + e] = s ? -v : v;
                }
                for_packed<NLOC, T, S>(static_cast<const S*>(A.pk), e0 + e, [&](int a, int q, T m) {
                    zl[a] = fma(m, xt[q * ne + e], zl[a]);
                    if (q < a) zl[q] = fma(m, xt[a * ne + e], zl[q]);
                });
            }
            __syncthreads();
            if (e < ne) {
#pragma unroll
                for (int a = 0; a < NLOC; ++a) {
                    // signs of the first 64 local dofs kept as bits, the rest re-read from loc
                    const bool s = a < 64 ? ((neg >> (a & 63)) & 1) != 0 : (loc[a * ne + e] & 0x8000) != 0;
                    zs[pos[a * ne + e]] = s ? -zl[a] : zl[a];
                }
            }
        } else {
            for (int it = tid; it < nitem; it += blockDim.x) {
                const int e = MR ? it / CW : it;
                const int rr = MR ? it % CW : 0;
                const uint16_t* L = loc + e;
                uint64_t neg = 0;
                T xl[NPAD];
#pragma unroll
                for (int a = 0; a < NLOC; ++a) {
                    const uint16_t c = L[a * ne];
                    if constexpr (SIGNED) {
                        const T v = (OP == OP_DIAG) ? T(0) : xs[(c & 0x7fff) * CW + rr];
                        const bool s = (c & 0x8000) != 0;
                        if (a < 64) neg |= (uint64_t)s << (a & 63);
                        xl[a] = s ? -v : v;
                    } else {
                        xl[a] = (OP == OP_DIAG) ? T(0) : xs[c * CW + rr];
                    }
                }
#pragma unroll
                for (int a = NLOC; a < NPAD; ++a) xl[a] = T(0);
                // the signed product v of copy (e, a): into its dof's accumulator (H1) or its
                // dof-sorted slot
                auto out = [&](int a, T v) {
                    if constexpr (FX) {
                        if constexpr (sizeof(T) == 4) acc.add_prescaled(L[a * ne] * CW + rr, v * scl);
                        else acc.add_scaled(L[a * ne] * CW + rr, v * sc);
                    } else {
                        const bool s = SIGNED && OP != OP_DIAG &&
                                       (a < 64 ? ((neg >> (a & 63)) & 1) != 0 : (L[a * ne] & 0x8000) != 0);
                        zs[pos[a * ne + e] * CW + rr] = s ? -v : v;
                    }
                };
                if constexpr (KIND == KIND_H1) {
                    using VM = typename Vec4<T>::type;
                    constexpr int W = Vec4<T>::W;
                    const T c = (MR || e != tid) ? static_cast<const T*>(A.scale)[e0 + e] : cfac;
#pragma unroll
                    for (int a = 0; a < NLOC; ++a) {
                        T accv = T(0);
                        if (OP == OP_DIAG) {
                            accv = Ms[a * NPAD + a];
                        } else {
                            const VM* row = reinterpret_cast<const VM*>(Ms + a * NPAD);
#pragma unroll
                            for (int q = 0; q < NPAD / W; ++q) {
                                const VM mm = row[q];
                                if constexpr (W == 4) {
                                    accv = fma(mm.x, xl[4 * q + 0], accv);
                                    accv = fma(mm.y, xl[4 * q + 1], accv);
                                    accv = fma(mm.z, xl[4 * q + 2], accv);
                                    accv = fma(mm.w, xl[4 * q + 3], accv);
                                } else {
                                    accv = fma(mm.x, xl[2 * q + 0], accv);
                                    accv = fma(mm.y, xl[2 * q + 1], accv);
                                }
                            }
                        }
                        out(a, accv * c);
                    }
                } else {
                    T zl[NLOC];
#pragma unroll
                    for (int a = 0; a < NLOC; ++a) zl[a] = T(0);
                    for_packed<NLOC, T, S>(static_cast<const S*>(A.pk), e0 + e, [&](int a, int q, T mm) {
                        if (OP == OP_DIAG) {
                            if (q == a) zl[a] = mm;
                        } else {
                            zl[a] = fma(mm, xl[q], zl[a]);
                            if (q < a) zl[q] = fma(mm, xl[a], zl[q]);
                        }
                    });
#pragma unroll
                    for (int a = 0; a < NLOC; ++a) out(a, zl[a]);
                }
            }
        }
        __syncthreads();

        if constexpr (FX) {
            // totals: interior dofs to y, shared ones to their partial slots
            for (int i = tid; i < nu * rc; i += blockDim.x) {
                const int u = i / rc, rr = i - u * rc;
                const T v = bad ? T(NAN) : fx_total(acc, u * CW + rr, kx, T(0));
                store_dof<T, OP, MR>(u, v, nint, ids, dmul, y, part, nrhs, r0 + rr, p0);
            }
        } else if constexpr (MR) {
            dof_run_sums<V>(nu, incoff, reinterpret_cast<const V*>(zs), vzero(V{}),
                            [](V a, const V& c) { return vsum(a, c); }, [&](int u, V v) {
                                if (u < nint) {
                                    if (OP == OP_BRAS) {
#pragma unroll
                                        for (int j = 0; j < CW; ++j) vget(v, j) = div_by_count(vget(v, j), dmul[u]);
                                    }
                                    st_seg(y + (size_t)ids[u] * nrhs + r0, rc, vec, v);
                                } else {
                                    st_seg(part + (size_t)(p0 + (u - nint)) * nrhs + r0, rc, vec, v);
                                }
                            });
        } else {
            dof_run_sums<T>(nu, incoff, zs, T(0), [](T a, T c) { return a + c; },
                            [&](int u, T v) { store_dof<T, OP, false>(u, v, nint, ids, dmul, y, part, nrhs, r0, p0); });
        }
        if (MR) __syncthreads();   // the sums are read before the next chunk stages x and clears
    }
}

template <int NLOC, typename T, int KIND>
size_t block_smem_bytes(const BlockArgs& A, bool mr = false) {
    constexpr int NPAD = PadTo<NLOC, T>::value;
    const size_t cw = mr ? Chunk<T>::CW : 1;
    const size_t xsb = sizeof(T) * (((size_t)A.max_u * cw + 3) & ~(size_t)3);
    if (KIND == KIND_H1)   // staged x, fixed-point accumulators, reference matrix
        return 128 + ((A.max_pkt + 127u) & ~127u) + xsb + 8 * (((size_t)A.max_u * cw + 1) & ~(size_t)1) +
               sizeof(T) * (size_t)NLOC * NPAD;
    // staged x, dof-sorted products
    return 128 + ((A.max_pkt + 127u) & ~127u) + xsb + sizeof(T) * (((size_t)NLOC * A.max_ne * cw + 3) & ~(size_t)3);
}

// ---- many right-hand sides, streamed cell matrices: cell products + dof gather -----------
// From kCellMrMinRhs right-hand sides on (n_loc <= 48), the apply runs as two kernels around a
// dof-sorted array of copies (the incidence-gather form of P^T):
//   k_cell_mr: one CTA per half tile of 16 cells (packet.h layout): the 16 cells' packed
//     matrices arrive in shared memory by bulk copies (one 256-byte run per 16-byte group), and
//     each warp takes (cell, 32 right-hand sides) items, lane = right-hand side: the local
//     vector and the accumulators stay in registers, every matrix group is one broadcast
//     shared-memory read for the 32 lanes, so each matrix byte feeds 32 right-hand sides; the
//     signed product a of cell e goes to its copy slot's row of R values;
//   k_dof_gather: y[u][r] = sum of dof u's copy rows in slot order (times 1/d for BRAS).
// Every sum has a fixed order: results are bit-reproducible.
constexpr int kCellMrMinRhs = 16;
constexpr int kCellMrMaxLoc = 48;  // local vector and accumulators in registers
constexpr int kCellMrCells = 16;   // cells of one CTA (half of a 32-cell tile)

template <int NLOC, typename S>
__host__ __device__ constexpr int mr_groups() {
    return (NLOC * (NLOC + 1) / 2 + PkVec<S>::G - 1) / PkVec<S>::G;
}
template <int NLOC, typename S>
constexpr size_t cell_mr_smem_bytes() {
    return 128 + (size_t)mr_groups<NLOC, S>() * kCellMrCells * 16;
}

template <int NLOC, typename T, typename S, int OP>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
k_cell_mr(const BlockArgs A, const T* __restrict__ x, T* __restrict__ cp, int R) {
    using V = typename PkVec<S>::V;
    constexpr int G = PkVec<S>::G, NG = mr_groups<NLOC, S>(), NC = kCellMrCells;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    const V* mat = reinterpret_cast<const V*>(smem_raw + 128);   // [g][cell] groups
    const int ht = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t e0 = (int64_t)ht * NC;
    const int ncell = (int)(A.n_cell - e0 < NC ? A.n_cell - e0 : NC);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {
        // group g of this half tile: NC * 16 contiguous bytes (the tile's 512-byte row g)
        const unsigned char* src = static_cast<const unsigned char*>(A.pk) +
                                   ((((size_t)(ht >> 1) * NG) << 5) + (size_t)(ht & 1) * NC) * 16;
        if (lane == 0) mbar_expect_tx(bar, (uint32_t)NG * NC * 16);
        __syncwarp();
        for (int g = lane; g < NG; g += 32)
            bulk_copy_g2s(smem_raw + 128 + (size_t)g * NC * 16, src + ((size_t)g << 5) * 16, NC * 16, bar);
    }
    const bool ok = cta_wait(bar, 0, A.status, true);
    if (!ok) {
        if (tid == 0) mbar_wait_bounded(bar, A.status);   // let the copies land before exiting
        return;
    }
    const T* dinv = static_cast<const T*>(A.dinv);
    const int nch = (R + 31) >> 5;
    for (int it = warp; it < ncell * nch; it += (int)(blockDim.x >> 5)) {
        const int c = it / nch;
        const int r = (it - c * nch) * 32 + lane;
        const bool act = r < R;
        const int64_t e = e0 + c;
        const int32_t* lg = A.mr_l2g + e * NLOC;
        T xl[NLOC], zl[NLOC];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            const int32_t gd = __ldg(lg + a);
            const int64_t u = gd & 0x7fffffff;
            T v = act ? __ldg(x + u * R + r) : T(0);
            if (OP == OP_BRAS) v *= __ldg(dinv + u);
            xl[a] = gd < 0 ? -v : v;
            zl[a] = T(0);
        }
        const V* mv = mat + c;
        int a = 0, q = 0;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const V v = mv[g * NC];
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (g * G + j < NLOC * (NLOC + 1) / 2) {
                    const T m = vec_elem<T>(v, j);
                    zl[a] = fma(m, xl[q], zl[a]);
                    if (q < a) zl[q] = fma(m, xl[a], zl[q]);
                    if (++q > a) {
                        ++a;
                        q = 0;
                    }
                }
            }
        }
        if (act) {
            const int32_t* sl = A.mr_slot + e * NLOC;
#pragma unroll
            for (int b = 0; b < NLOC; ++b) {
                const T v = __ldg(lg + b) < 0 ? -zl[b] : zl[b];
                cp[(int64_t)__ldg(sl + b) * R + r] = v;
            }
        }
    }
}

// The same with FP64 vectors and float-float cell products (the refinement residual b - M x of
// the mixed solve on many right-hand sides): M_K as (hi, lo) float pairs, x split once per
// value, every product term compensated (df_term, about 2^-48), each result rounded to FP64
// once.  B300 runs FP64 arithmetic at 1/64 of the FP32 rate; this runs on the FP32 units.
template <int NLOC>
__global__ void __launch_bounds__(256, 1)
k_cell_mr_df(const BlockArgs A, const double* __restrict__ x, double* __restrict__ cp, int R) {
    constexpr int NPK = NLOC * (NLOC + 1) / 2, NG = (NPK + 1) / 2, NC = kCellMrCells;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    const float4* mat = reinterpret_cast<const float4*>(smem_raw + 128);   // [g][cell]: two (hi, lo) entries
    const int ht = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t e0 = (int64_t)ht * NC;
    const int ncell = (int)(A.n_cell - e0 < NC ? A.n_cell - e0 : NC);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned char* src = reinterpret_cast<const unsigned char*>(A.pk_df) +
                                   ((((size_t)(ht >> 1) * NG) << 5) + (size_t)(ht & 1) * NC) * 16;
        if (lane == 0) mbar_expect_tx(bar, (uint32_t)NG * NC * 16);
        __syncwarp();
        for (int g = lane; g < NG; g += 32)
            bulk_copy_g2s(smem_raw + 128 + (size_t)g * NC * 16, src + ((size_t)g << 5) * 16, NC * 16, bar);
    }
    if (!cta_wait(bar, 0, A.status, true)) {
        if (tid == 0) mbar_wait_bounded(bar, A.status);
        return;
    }
    const int nch = (R + 31) >> 5;
    for (int it = warp; it < ncell * nch; it += (int)(blockDim.x >> 5)) {
        const int c = it / nch;
        const int r = (it - c * nch) * 32 + lane;
        const bool act = r < R;
        const int64_t e = e0 + c;
        const int32_t* lg = A.mr_l2g + e * NLOC;
        float xh[NLOC], xl[NLOC], zh[NLOC], zl[NLOC];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            const int32_t gd = __ldg(lg + a);
            double v = act ? __ldg(x + (int64_t)(gd & 0x7fffffff) * R + r) : 0.0;
            if (gd < 0) v = -v;
            xh[a] = (float)v;
            xl[a] = (float)(v - (double)xh[a]);
            zh[a] = zl[a] = 0.f;
        }
        const float4* mv = mat + c;
        int a = 0, q = 0;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const float4 v = mv[g * NC];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (2 * g + j < NPK) {
                    const float mh = j ? v.z : v.x, ml = j ? v.w : v.y;
                    df_term(mh, ml, xh[q], xl[q], zh[a], zl[a]);
                    if (q < a) df_term(mh, ml, xh[a], xl[a], zh[q], zl[q]);
                    if (++q > a) {
                        ++a;
                        q = 0;
                    }
                }
            }
        }
        if (act) {
            const int32_t* sl = A.mr_slot + e * NLOC;
#pragma unroll
            for (int b = 0; b < NLOC; ++b) {
                const double v = (double)zh[b] + (double)zl[b];
                cp[(int64_t)__ldg(sl + b) * R + r] = __ldg(lg + b) < 0 ? -v : v;
            }
        }
    }
}

// One thread per (dof, rhs): consecutive threads take consecutive right-hand sides of a dof,
// so every copy row is one coalesced read; a dof's first four copies are loaded together (more
// bytes in flight per thread), and each dof adds its copies in slot order.
template <typename T, int OP>
__global__ void __launch_bounds__(256) k_dof_gather(const BlockArgs A, const T* __restrict__ cp, T* __restrict__ y,
                                                    int R) {
    constexpr int C = 4;
    const int64_t total = A.n_dof * R;
    const T* dinv = static_cast<const T*>(A.dinv);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i / R;
        const int r = (int)(i - u * R);
        const int64_t s0 = __ldg(A.mr_off + u), s1 = __ldg(A.mr_off + u + 1);
        const T* row = cp + s0 * R + r;
        const int64_t cnt = s1 - s0;
        T v[C];
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = j < cnt ? __ldg(row + (int64_t)j * R) : T(0);
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (j < cnt) acc += v[j];
        for (int64_t j = C; j < cnt; ++j) acc += __ldg(row + j * R);
        y[i] = (OP == OP_BRAS) ? acc * __ldg(dinv + u) : acc;
    }
}

template <int NLOC, typename T, typename S, int OP>
cudaError_t launch_cell_mr(const BlockArgs& A, const T* x, T* y, T* cp, int nrhs, cudaStream_t st) {
    auto kern = k_cell_mr<NLOC, T, S, OP>;
    const size_t smem = cell_mr_smem_bytes<NLOC, S>();
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int nct = (int)((A.n_cell + kCellMrCells - 1) / kCellMrCells);
    kern<<<nct, 256, smem, st>>>(A, x, cp, nrhs);
    count_launch(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int nb = (int)std::min<int64_t>((A.n_dof * nrhs + 255) / 256, 148 * 16);
    k_dof_gather<T, OP><<<nb, 256, 0, st>>>(A, cp, y, nrhs);
    count_launch(1);
    return cudaGetLastError();
}

template <int NLOC>
cudaError_t launch_cell_mr_df(const BlockArgs& A, const double* x, double* y, double* cp, int nrhs, cudaStream_t st) {
    auto kern = k_cell_mr_df<NLOC>;
    const size_t smem = 128 + (size_t)((NLOC * (NLOC + 1) / 2 + 1) / 2) * kCellMrCells * 16;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int nct = (int)((A.n_cell + kCellMrCells - 1) / kCellMrCells);
    kern<<<nct, 256, smem, st>>>(A, x, cp, nrhs);
    count_launch(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int nb = (int)std::min<int64_t>((A.n_dof * nrhs + 255) / 256, 148 * 16);
    k_dof_gather<double, OP_MASS><<<nb, 256, 0, st>>>(A, cp, y, nrhs);
    count_launch(1);
    return cudaGetLastError();
}

// The many-right-hand-side path applies (kernel family, n_loc, call)
template <int NLOC, int KIND, int OP>
__host__ __device__ constexpr bool cell_mr_kind() {
    return KIND == KIND_PACKED && NLOC <= kCellMrMaxLoc && OP != OP_DIAG;
}
inline bool cell_mr_call(const BlockArgs& A, int nrhs) { return A.mr_l2g != nullptr && nrhs >= kCellMrMinRhs; }

// Largest dynamic shared memory one CTA may opt into on the current device.
int smem_optin_bytes();
// Shared memory of one SM of the current device.
int smem_per_sm_bytes();

// Rows of nrhs values 16-byte aligned, so that full chunks load and store as one vector.
template <typename T>
inline bool rows_vectorisable(int nrhs, const void* x, const void* y, const void* part) {
    const int per16 = 16 / (int)sizeof(T);
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return nrhs % per16 == 0 && al(x) && al(y) && al(part);
}

// Launch one block apply (block kernel + combine pass).  Returns a cudaError_t.  Several right-hand sides go
// to the multi-RHS kernel when its chunk buffers fit shared memory, else to one CTA per
// (block, rhs).
template <int NLOC, typename T, typename S, int KIND, int OP>
cudaError_t launch_block(const BlockArgs& A, const CombineArgs& G, int nblk, const T* x, T* y, T* part, int nrhs,
                         cudaStream_t st) {
    // multi-RHS items hold their local vector and accumulators in registers: n_loc <= 48
    if constexpr (cell_mr_kind<NLOC, KIND, OP>()) {
        if (cell_mr_call(A, nrhs)) {
            if constexpr (sizeof(T) == 8 && OP == OP_MASS) {
                if (A.pk_df) return launch_cell_mr_df<NLOC>(A, x, y, part, nrhs, st);
            }
            return launch_cell_mr<NLOC, T, S, OP>(A, x, y, part, nrhs, st);
        }
    }
    constexpr bool kMR = NLOC <= 48;
    const bool mr = kMR && nrhs > 1 && OP != OP_DIAG &&
                    block_smem_bytes<NLOC, T, KIND>(A, true) <= (size_t)smem_optin_bytes();
    const size_t smem = block_smem_bytes<NLOC, T, KIND>(A, mr);
    auto kern = k_block<NLOC, T, S, KIND, OP, false>;
    if constexpr (kMR) {
        if (mr) kern = k_block<NLOC, T, S, KIND, OP, true>;
    }
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err != cudaSuccess) return err;
    dim3 grid(mr ? nblk : nblk * nrhs);
    // one thread per cell of the largest block (at most 256: larger H1 blocks loop over their
    // cells); multi-RHS: 256 threads over the block's items
    const int threads = mr ? 256 : std::min(256, (A.max_ne + 31) / 32 * 32);
    const int vec = rows_vectorisable<T>(nrhs, x, y, part) ? 1 : 0;
    err = launch_pdl(kern, grid, dim3(threads), smem, st, A, x, y, part, nrhs, vec);
    count_launch(1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_group_combine<T, OP>(G, part, A.npart, y, nrhs, mr, st);
}

}  // namespace bras
