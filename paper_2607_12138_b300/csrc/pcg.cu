// Preconditioned CG mass solve (Sec. 3) and FP64 iterative refinement around an FP32 inner
// solve.  Dot products accumulate in FP64 through a fixed two-level tree (per-block partial
// sums, then one block summing them in block order): results are bit-reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "internal.h"

namespace bras {

constexpr int kDotBlocks = 1184;   // at most 8 per SM on a 148-SM B300 (the partial-sum buffer)
constexpr int kMaxRhs = 256;

// per-slot scalars; S_BN, S_RN = ||b||, ||b - M x|| of the refinement loop
enum { S_RZ = 0, S_PQ, S_RR, S_RR0, S_ALPHA, S_BETA, S_ISCALE, S_SCALE, S_BN, S_RN, S_COUNT };
enum { FIN_INIT_RR = 0, FIN_INIT_RZ, FIN_ALPHA, FIN_RR, FIN_BETA, FIN_NORM,
       // stationary iterations: as FIN_INIT_RR / FIN_RR, then the step of the next update is
       // sc[S_SCALE] for an active rhs and 0 for a converged one
       FIN_INIT_STAT, FIN_RR_STAT,
       // power iteration: store the dot product in S_RZ / S_PQ
       FIN_STORE_A, FIN_STORE_B,
       // refinement loop: (b, b) and (r, r) of the true residual -> scales, inner tolerance,
       // outer loop condition; FIN_INIT_INNER = FIN_INIT_RR + the inner loop condition
       FIN_OUTER_INIT, FIN_OUTER, FIN_INIT_INNER };
enum { SOLVER_CG = 0, SOLVER_FIXED_POINT = 1, SOLVER_CHEBYSHEV = 2, SOLVER_MIXED = 3 };
constexpr int kMaxOuter = 60;      // refinement steps of a mixed solve at most
// iparam: [0] inner maxit, [1] inner iterations done, [2] maxit of the whole mixed solve,
// [3] inner iterations charged so far (at least 1 per refinement step), [4] refinement steps
// done, [5] outer loop condition, [6] inner loop condition, [7] inner iterations done in all
enum { IP_MAXIT = 0, IP_DONE, IP_MAXIT_ALL, IP_CHARGED, IP_OUTER, IP_GO_OUTER, IP_GO_INNER, IP_DONE_ALL, IP_COUNT };

struct SolveGraph {
    int solver = SOLVER_CG, prec = 0, pc = 0, R = 0, tsize = 0;
    const void *x = nullptr, *part = nullptr;
    const void* coef = nullptr;   // Chebyshev coefficient table captured in the body
    int coef_k = 0;
    int kernels_per_iter = 0;
    int mixed_init = 0, mixed_start = 0, mixed_post = 0;   // mixed solve: kernels of its other parts
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct PcgWork {
    cudaStream_t cap = nullptr;   // private stream used only to capture solve graphs
    std::vector<SolveGraph> graphs;
    double* dparam = nullptr;     // [0] = rtol^2 of the CG loop, [1] = rtol of a mixed solve
    int* iparam = nullptr;        // [IP_COUNT], see IP_*
    double* h_param = nullptr;    // pinned staging of dparam/iparam
    int nrhs = 0;
    int slots = 0;                // scalar slots: max(nrhs, meshes of a batch)
    int64_t n = 0;
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *xs = nullptr, *bs = nullptr;
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *x32 = nullptr;
    double* partial = nullptr;    // [kDotBlocks][nrhs]
    unsigned int* ticket = nullptr;  // arrival counter of the fused reductions
    double* sc = nullptr;         // [S_COUNT][nrhs]
    int* flags = nullptr;         // [0..S): active, [S..2S): its, [2S]: n active, [2S+1]: status,
                                  // [2S+2..3S+2): inner iterations of a mixed solve (S = slots)
    int* h_flags = nullptr;       // pinned
    double* h_sc = nullptr;       // pinned
    double* coef = nullptr;       // Chebyshev direction coefficients [2][kmax + 1][slots]
    int coef_k = 0;               // kmax of the allocation
    double* hist = nullptr;       // CG-Lanczos: alpha_k, beta_k of rhs 0 ([2][hist_cap]); null otherwise
    int hist_cap = 0;
};

void free_pcg(bras_ctx* c) {
    if (!c->pcg) return;
    for (auto& g : c->pcg->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    c->pcg->graphs.clear();
    if (c->pcg->cap) cudaStreamDestroy(c->pcg->cap);
    if (c->pcg->h_param) cudaFreeHost(c->pcg->h_param);
    if (c->pcg->h_flags) cudaFreeHost(c->pcg->h_flags);
    if (c->pcg->h_sc) cudaFreeHost(c->pcg->h_sc);
    delete c->pcg;       // device buffers are in c->owned
    c->pcg = nullptr;
}

static int ensure_pcg(bras_ctx* c, int R, bool mixed) {
    PcgWork* w = c->pcg;
    if (w && w->nrhs >= R && (!mixed || w->r32)) return BRAS_OK;
    if (w) {
        for (void* p : {(void*)w->r, (void*)w->z, (void*)w->p, (void*)w->q, (void*)w->xs, (void*)w->bs,
                        (void*)w->r32, (void*)w->z32, (void*)w->p32, (void*)w->q32, (void*)w->x32,
                        (void*)w->partial, (void*)w->sc, (void*)w->flags, (void*)w->dparam, (void*)w->iparam, (void*)w->ticket,
                        (void*)w->coef})
            dfree(c, p);
        free_pcg(c);
    }
    w = new PcgWork();
    c->pcg = w;
    w->nrhs = std::max(R, c->max_nrhs);
    w->n = c->n;
    const size_t nv = (size_t)c->n * w->nrhs;
    auto d = [&](size_t b) { return dalloc_bytes(c, b); };
    w->r = (double*)d(nv * 8);
    w->z = (double*)d(nv * 8);
    w->p = (double*)d(nv * 8);
    w->q = (double*)d(nv * 8);
    w->xs = (double*)d(nv * 8);
    w->bs = (double*)d(nv * 8);
    const size_t slots = (size_t)std::max(w->nrhs, c->n_mesh);
    w->slots = (int)slots;
    w->partial = (double*)d(std::max((size_t)kDotBlocks * w->nrhs, (size_t)c->nseg) * 8);
    w->sc = (double*)d((size_t)S_COUNT * slots * 8);
    w->flags = (int*)d((3 * slots + 2) * 4);
    w->dparam = (double*)d(8 * 2);
    w->ticket = (unsigned int*)d(16);
    if (!w->ticket || cudaMemset(w->ticket, 0, 16) != cudaSuccess) return BRAS_ERR_OOM;
    w->iparam = (int*)d(4 * IP_COUNT);
    if (!w->dparam || !w->iparam) return BRAS_ERR_OOM;
    if (cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking) != cudaSuccess) return BRAS_ERR_CUDA;
    if (cudaMallocHost(&w->h_param, 16 + 4 * IP_COUNT) != cudaSuccess) return BRAS_ERR_OOM;
    if (!w->r || !w->z || !w->p || !w->q || !w->xs || !w->bs || !w->partial || !w->sc || !w->flags) return BRAS_ERR_OOM;
    if (mixed) {
        w->r32 = (float*)d(nv * 4);
        w->z32 = (float*)d(nv * 4);
        w->p32 = (float*)d(nv * 4);
        w->q32 = (float*)d(nv * 4);
        w->x32 = (float*)d(nv * 4);
        if (!w->r32 || !w->z32 || !w->p32 || !w->q32 || !w->x32) return BRAS_ERR_OOM;
    }
    if (cudaMallocHost(&w->h_flags, (3 * slots + 2) * sizeof(int)) != cudaSuccess) return BRAS_ERR_OOM;
    if (cudaMallocHost(&w->h_sc, S_COUNT * slots * sizeof(double)) != cudaSuccess) return BRAS_ERR_OOM;
    return BRAS_OK;
}

// ---- kernels ---------------------------------------------------------------------------
// Every dot product ends in a fixed-order two-level reduction: each block writes its partial
// sum, takes a ticket (an integer atomic, so the order of arrival does not matter), and the
// last block to arrive reduces all partials in a fixed tree order and applies the scalar
// update of the CG step (alpha, beta, convergence masks, loop condition).  No floating-point
// atomics; results are bit-reproducible.
struct FinArgs {
    int kind;
    double* partial;               // [G][R] per-block partial sums
    unsigned int* ticket;          // arrival counter, returned to 0 by the last block
    double* sc;                    // per-rhs scalars [S_COUNT][R]
    int* flags;                    // active[R], its[R], n_active, status
    double* dparam;                // [0] = rtol^2 of the CG loop, [1] = rtol of a mixed solve
    int* iparam;                   // [0] = maxit, [1] = iterations done
    cudaGraphConditionalHandle cond;
    int in_graph;                  // the loop condition exists (solve graph)
    double* hist;                  // if set: alpha_k -> hist[k], beta_k -> hist[cap + k] (slot 0)
    int hist_cap;
};

__device__ void apply_fin(const FinArgs& F, int R, int r, double s) {
    double* sc = F.sc;
    int* active = F.flags;
    int* its = F.flags + R;
    const double tol2 = F.dparam ? F.dparam[0] : 0.0;
    switch (F.kind) {
        case FIN_INIT_RR:
            sc[S_RR0 * R + r] = s;
            sc[S_RR * R + r] = s;
            active[r] = s > 0.0 ? 1 : 0;
            its[r] = 0;
            break;
        case FIN_INIT_RZ:
            sc[S_RZ * R + r] = s;
            break;
        case FIN_ALPHA: {
            sc[S_PQ * R + r] = s;
            double a = 0.0;
            if (active[r]) {
                if (!(s > 0.0) || !isfinite(s)) {
                    active[r] = 0;
                    F.flags[2 * R + 1] = BRAS_ERR_BREAKDOWN;
                } else {
                    a = sc[S_RZ * R + r] / s;
                }
            }
            sc[S_ALPHA * R + r] = a;
            if (F.hist && r == 0 && active[r] && its[r] < F.hist_cap) F.hist[its[r]] = a;
            break;
        }
        case FIN_RR:
            sc[S_RR * R + r] = s;
            if (active[r]) {
                its[r] += 1;
                if (s <= tol2 * sc[S_RR0 * R + r]) active[r] = 0;
            }
            break;
        case FIN_BETA: {   // beta = 0 on the first iteration (p = z)
            double bta = 0.0;
            if (active[r]) {
                bta = its[r] == 0 ? 0.0 : s / sc[S_RZ * R + r];
                sc[S_RZ * R + r] = s;
                if (F.hist && r == 0 && its[r] < F.hist_cap) F.hist[F.hist_cap + its[r]] = bta;
            }
            sc[S_BETA * R + r] = bta;
            break;
        }
        case FIN_NORM:
            sc[S_RR * R + r] = s;
            break;
        case FIN_INIT_STAT:
            sc[S_RR0 * R + r] = s;
            sc[S_RR * R + r] = s;
            active[r] = s > 0.0 ? 1 : 0;
            its[r] = 0;
            sc[S_ALPHA * R + r] = active[r] ? sc[S_SCALE * R + r] : 0.0;
            break;
        case FIN_RR_STAT:
            sc[S_RR * R + r] = s;
            if (active[r]) {
                its[r] += 1;
                if (!isfinite(s)) {
                    active[r] = 0;
                    F.flags[2 * R + 1] = BRAS_ERR_BREAKDOWN;
                } else if (s <= tol2 * sc[S_RR0 * R + r]) {
                    active[r] = 0;
                }
            }
            sc[S_ALPHA * R + r] = active[r] ? sc[S_SCALE * R + r] : 0.0;
            break;
        case FIN_STORE_A:
            sc[S_RZ * R + r] = s;
            break;
        case FIN_STORE_B:
            sc[S_PQ * R + r] = s;
            break;
        case FIN_INIT_INNER:
            sc[S_RR0 * R + r] = s;
            sc[S_RR * R + r] = s;
            active[r] = s > 0.0 ? 1 : 0;
            its[r] = 0;
            break;
        case FIN_OUTER_INIT:
        case FIN_OUTER: {
            // s = ||b||^2 (init) or ||b - M x||^2; a slot is refined while ||r|| / ||b|| > rtol,
            // its inner right-hand side is r / ||r|| and the inner solution is added times ||r||
            int* its_all = F.flags + 2 * R + 2;
            const double rn = sqrt(s);
            double bn;
            if (F.kind == FIN_OUTER_INIT) {
                bn = rn;
                sc[S_BN * R + r] = bn;
                its_all[r] = 0;
            } else {
                bn = sc[S_BN * R + r];
                its_all[r] += its[r];
            }
            sc[S_RN * R + r] = rn;
            const double rel = bn > 0.0 ? rn / bn : 0.0;
            const bool refine = bn > 0.0 && rel > F.dparam[1];
            sc[S_SCALE * R + r] = refine ? 1.0 / rn : 0.0;
            sc[S_ISCALE * R + r] = refine ? rn : 0.0;
            break;
        }
    }
}

__device__ __forceinline__ bool fin_counts_iteration(int kind) { return kind == FIN_RR || kind == FIN_RR_STAT; }

// Scalar tail of a fused reduction, run by one thread after every slot's apply_fin: the
// count of active slots `cnt`, iteration counting and the loop conditions.
__device__ void fin_tail(const FinArgs& F, int R, int cnt) {
    F.flags[2 * R] = cnt;
    int* ip = F.iparam;
    if (fin_counts_iteration(F.kind) && ip) {
        const int done = ++ip[IP_DONE];
        const unsigned go = (cnt > 0 && done < ip[IP_MAXIT]) ? 1u : 0u;
        ip[IP_GO_INNER] = (int)go;
        if (F.in_graph) cudaGraphSetConditional(F.cond, go);
    }
    if (F.kind == FIN_INIT_INNER && ip) {
        ip[IP_DONE] = 0;
        const unsigned go = (cnt > 0 && ip[IP_MAXIT] > 0) ? 1u : 0u;
        ip[IP_GO_INNER] = (int)go;
        if (F.in_graph) cudaGraphSetConditional(F.cond, go);
    }
    if ((F.kind == FIN_OUTER_INIT || F.kind == FIN_OUTER) && ip) {
        double worst = 0.0;
        for (int k = 0; k < R; ++k) {
            const double bn = F.sc[S_BN * R + k];
            const double rel = bn > 0.0 ? F.sc[S_RN * R + k] / bn : 0.0;
            if (rel > worst) worst = rel;
        }
        int charged = 0, outer = 0;
        if (F.kind == FIN_OUTER) {
            charged = ip[IP_CHARGED] + max(ip[IP_DONE], 1);
            outer = ip[IP_OUTER] + 1;
            ip[IP_DONE_ALL] += ip[IP_DONE];
        } else {
            ip[IP_DONE_ALL] = 0;
        }
        ip[IP_CHARGED] = charged;
        ip[IP_OUTER] = outer;
        const double rtol = F.dparam[1];
        const unsigned go =
            (worst > rtol && charged < ip[IP_MAXIT_ALL] && outer < kMaxOuter && F.flags[2 * R + 1] == 0) ? 1u : 0u;
        // inner tolerance: as deep as FP32 allows, no deeper than the outer test needs
        const double tin = fmax(1e-6, fmin(1e-2, 0.5 * rtol / worst));
        F.dparam[0] = tin * tin;
        ip[IP_MAXIT] = ip[IP_MAXIT_ALL] - charged;
        ip[IP_GO_OUTER] = (int)go;
        if (F.in_graph) cudaGraphSetConditional(F.cond, go);
    }
}

// `red` holds this block's 256 per-thread sums (thread t: rhs t % R, group t / R).
// Fixed-order sum of a 256-thread block's values (one right-hand side): a shuffle tree within
// each warp, then the eight warp sums in warp order.  Every thread gets the total.
__device__ __forceinline__ double block_sum_fixed(double v, double* wsum) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += wsum[w];
    return s;
}

__device__ void block_partial_and_finish(const FinArgs& F, int R, double* red) {
    const int tid = threadIdx.x, J = 256 / R, r = tid % R, j = tid / R;
    __shared__ unsigned int s_last;
    if (R == 1) {
        // one right-hand side: shuffle trees instead of the shared-memory tree
        __shared__ double wsum[8];
        const double bs = block_sum_fixed(red[tid], wsum);
        if (tid == 0) {
            F.partial[blockIdx.x] = bs;
            __threadfence();
            s_last = (atomicAdd(F.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        double v = 0.0;
        for (int g = tid; g < (int)gridDim.x; g += 256) v += __ldcg(&F.partial[g]);
        __syncthreads();   // wsum is reused
        const double total = block_sum_fixed(v, wsum);
        if (tid == 0) {
            apply_fin(F, 1, 0, total);
            fin_tail(F, 1, F.flags[0]);
            *F.ticket = 0u;
        }
        return;
    }
    // fixed tree over the J groups of this block
    for (int h = 1; h < J; h *= 2) {
        __syncthreads();
        if (j < J && (j % (2 * h)) == 0 && j + h < J) red[tid] += red[tid + h * R];
    }
    __syncthreads();
    if (tid < R) F.partial[blockIdx.x * R + tid] = red[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(F.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: fixed-order reduction of all G partials
    double s = 0.0;
    if (j < J)
        for (int g = j; g < (int)gridDim.x; g += J) s += __ldcg(&F.partial[g * R + r]);
    red[tid] = s;
    for (int h = 1; h < J; h *= 2) {
        __syncthreads();
        if (j < J && (j % (2 * h)) == 0 && j + h < J) red[tid] += red[tid + h * R];
    }
    __syncthreads();
    if (tid < R) apply_fin(F, R, tid, red[tid]);
    __syncthreads();
    if (tid == 0) {
        int cnt = 0;
        for (int k = 0; k < R; ++k) cnt += F.flags[k];
        fin_tail(F, R, cnt);
        *F.ticket = 0u;
    }
}

// Per-thread sums of products.  FP64 vectors: FP64 products and sums.  FP32 vectors: the
// products are formed exactly (p + e = a b by an FMA) and summed as float-float pairs with a
// two-sum (about 2^-48 relative per step, like an FP64 sum) on the FP32 units -- B300 issues
// FP64 at 1/64 of the FP32 rate -- and each thread's pair is finished in FP64 for the
// fixed-order block and grid reductions.
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        const float t = __fadd_rn(h, p);
        const float bp = __fsub_rn(t, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        h = t;
        l = __fadd_rn(l, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};
template <typename TA, typename TB> struct DotType { using type = double; };
template <> struct DotType<float, float> { using type = float; };

// Thread t of a block handles rhs t % R of rows t / R, so every thread sticks to one rhs.
// One right-hand side with 16-byte aligned vectors (vec): 16-byte loads, four in flight per
// array and thread, the n mod W last values taken one each by the first threads.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_dot(const TA* __restrict__ a, const TB* __restrict__ b, int64_t n, int R,
                                             int vec, FinArgs F) {
    using TD = typename DotType<TA, TB>::type;
    __shared__ double red[256];
    pdl_launch();
    pdl_wait();
    const int rows = 256 / R, tid = threadIdx.x, r = tid % R, lr = tid / R;
    double acc = 0.0;
    if constexpr (std::is_same<TA, TB>::value) {
        if (vec) {
            using V = typename Vec4<TA>::type;
            constexpr int W = Vec4<TA>::W;
            const V* av = reinterpret_cast<const V*>(a);
            const V* bv = reinterpret_cast<const V*>(b);
            const int64_t nvec = n / W, stride = (int64_t)gridDim.x * 256;
            const int64_t gid = (int64_t)blockIdx.x * 256 + tid;
            DotAcc<TD> c[4];
            int64_t i = gid;
            for (; i + 3 * stride < nvec; i += 4 * stride) {
                V x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    x[u] = av[i + u * stride];
                    y[u] = bv[i + u * stride];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int j = 0; j < W; ++j) c[u].add((TD)vget(x[u], j), (TD)vget(y[u], j));
            }
            for (; i < nvec; i += stride) {
                V x = av[i], y = bv[i];
#pragma unroll
                for (int j = 0; j < W; ++j) c[0].add((TD)vget(x, j), (TD)vget(y, j));
            }
            if (gid < n - nvec * W) c[1].add((TD)a[nvec * W + gid], (TD)b[nvec * W + gid]);
            red[tid] = (c[0].value() + c[1].value()) + (c[2].value() + c[3].value());
            block_partial_and_finish(F, 1, red);
            return;
        }
    }
    if (lr < rows) {
        // four independent accumulators (loads in flight), combined in a fixed order
        const int64_t stride = (int64_t)gridDim.x * rows;
        int64_t i = (int64_t)blockIdx.x * rows + lr;
        DotAcc<TD> c0, c1, c2, c3;
        for (; i + 3 * stride < n; i += 4 * stride) {
            c0.add((TD)a[i * R + r], (TD)b[i * R + r]);
            c1.add((TD)a[(i + stride) * R + r], (TD)b[(i + stride) * R + r]);
            c2.add((TD)a[(i + 2 * stride) * R + r], (TD)b[(i + 2 * stride) * R + r]);
            c3.add((TD)a[(i + 3 * stride) * R + r], (TD)b[(i + 3 * stride) * R + r]);
        }
        for (; i < n; i += stride) c0.add((TD)a[i * R + r], (TD)b[i * R + r]);
        acc = (c0.value() + c1.value()) + (c2.value() + c3.value());
    }
    red[tid] = acc;
    block_partial_and_finish(F, R, red);
}

// x += alpha p; r -= alpha q; and r.r with the convergence test  (fused, one pass; vec: one
// right-hand side, 16-byte aligned vectors, 16-byte accesses as in k_dot)
template <typename T>
__global__ void __launch_bounds__(256) k_update_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                   const T* __restrict__ q, const double* __restrict__ alpha,
                                                   int64_t n, int R, int vec, FinArgs F) {
    __shared__ double red[256];
    pdl_launch();
    pdl_wait();
    const int rows = 256 / R, tid = threadIdx.x, rr = tid % R, lr = tid / R;
    double acc = 0.0;
    if (vec) {
        using V = typename Vec4<T>::type;
        constexpr int W = Vec4<T>::W;
        const T a = (T)alpha[0];
        V* xv = reinterpret_cast<V*>(x);
        V* rv = reinterpret_cast<V*>(r);
        const V* pv = reinterpret_cast<const V*>(p);
        const V* qv = reinterpret_cast<const V*>(q);
        const int64_t nvec = n / W, stride = (int64_t)gridDim.x * 256;
        const int64_t gid = (int64_t)blockIdx.x * 256 + tid;
        DotAcc<T> c[4];
        int64_t i = gid;
        for (; i + 3 * stride < nvec; i += 4 * stride) {
            V pp[4], qq[4], xx[4], ro[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                pp[u] = pv[i + u * stride];
                qq[u] = qv[i + u * stride];
                xx[u] = xv[i + u * stride];
                ro[u] = rv[i + u * stride];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    vget(xx[u], j) = fma(a, vget(pp[u], j), vget(xx[u], j));
                    const T v = fma(-a, vget(qq[u], j), vget(ro[u], j));
                    vget(ro[u], j) = v;
                    c[u].add(v, v);
                }
                xv[i + u * stride] = xx[u];
                rv[i + u * stride] = ro[u];
            }
        }
        for (; i < nvec; i += stride) {
            V pp = pv[i], qq = qv[i], xx = xv[i], ro = rv[i];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                vget(xx, j) = fma(a, vget(pp, j), vget(xx, j));
                const T v = fma(-a, vget(qq, j), vget(ro, j));
                vget(ro, j) = v;
                c[0].add(v, v);
            }
            xv[i] = xx;
            rv[i] = ro;
        }
        if (gid < n - nvec * W) {
            const int64_t k = nvec * W + gid;
            x[k] = fma(a, p[k], x[k]);
            const T v = fma(-a, q[k], r[k]);
            r[k] = v;
            c[1].add(v, v);
        }
        red[tid] = (c[0].value() + c[1].value()) + (c[2].value() + c[3].value());
        block_partial_and_finish(F, 1, red);
        return;
    }
    if (lr < rows) {
        const T a = (T)alpha[rr];
        const int64_t stride = (int64_t)gridDim.x * rows;
        int64_t i = (int64_t)blockIdx.x * rows + lr;
        DotAcc<T> c[4];
        for (; i + 3 * stride < n; i += 4 * stride) {
            T pv[4], qv[4], xv[4], rv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = (i + u * stride) * R + rr;
                pv[u] = p[k];
                qv[u] = q[k];
                xv[u] = x[k];
                rv[u] = r[k];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = (i + u * stride) * R + rr;
                x[k] = fma(a, pv[u], xv[u]);
                const T v = fma(-a, qv[u], rv[u]);
                r[k] = v;
                c[u].add(v, v);
            }
        }
        for (; i < n; i += stride) {
            const int64_t k = i * R + rr;
            x[k] = fma(a, p[k], x[k]);
            const T v = fma(-a, q[k], r[k]);
            r[k] = v;
            c[0].add(v, v);
        }
        acc = (c[0].value() + c[1].value()) + (c[2].value() + c[3].value());
    }
    red[tid] = acc;
    block_partial_and_finish(F, R, red);
}

// ---- refinement loop of the mixed solve (one graph: the outer loop and the inner CG loop are
// conditional WHILE nodes; these kernels end in the fused reductions that decide them) ------
// x = 0; r = b; (b, b) -> FIN_OUTER_INIT
__global__ void __launch_bounds__(256) k_outer_init(double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ b, int64_t n, int R, FinArgs F) {
    __shared__ double red[256];
    const int rows = 256 / R, tid = threadIdx.x, rr = tid % R, lr = tid / R;
    double acc = 0.0;
    if (lr < rows) {
        const int64_t stride = (int64_t)gridDim.x * rows;
        DotAcc<double> c[4];
        int64_t i = (int64_t)blockIdx.x * rows + lr;
        for (; i + 3 * stride < n; i += 4 * stride) {
            double bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) bv[u] = b[(i + u * stride) * R + rr];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = (i + u * stride) * R + rr;
                r[k] = bv[u];
                x[k] = 0.0;
                c[u].add(bv[u], bv[u]);
            }
        }
        for (; i < n; i += stride) {
            const int64_t k = i * R + rr;
            const double v = b[k];
            r[k] = v;
            x[k] = 0.0;
            c[0].add(v, v);
        }
        acc = (c[0].value() + c[1].value()) + (c[2].value() + c[3].value());
    }
    red[tid] = acc;
    block_partial_and_finish(F, R, red);
}

// inner start: r32 = (float)(r s) (s = 1/||r|| or 0), x32 = p32 = 0; (r32, r32) -> FIN_INIT_INNER
__global__ void __launch_bounds__(256) k_inner_start(const double* __restrict__ r, const double* __restrict__ s,
                                                    float* __restrict__ r32, float* __restrict__ x32,
                                                    float* __restrict__ p32, int64_t n, int R, FinArgs F) {
    __shared__ double red[256];
    const int rows = 256 / R, tid = threadIdx.x, rr = tid % R, lr = tid / R;
    double acc = 0.0;
    if (lr < rows) {
        const double sc = s[rr];
        const int64_t stride = (int64_t)gridDim.x * rows;
        DotAcc<float> c[4];
        int64_t i = (int64_t)blockIdx.x * rows + lr;
        for (; i + 3 * stride < n; i += 4 * stride) {
            double rv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) rv[u] = r[(i + u * stride) * R + rr];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = (i + u * stride) * R + rr;
                const float v = (float)(rv[u] * sc);
                r32[k] = v;
                x32[k] = 0.f;
                p32[k] = 0.f;
                c[u].add(v, v);
            }
        }
        for (; i < n; i += stride) {
            const int64_t k = i * R + rr;
            const float v = (float)(r[k] * sc);
            r32[k] = v;
            x32[k] = 0.f;
            p32[k] = 0.f;
            c[0].add(v, v);
        }
        acc = (c[0].value() + c[1].value()) + (c[2].value() + c[3].value());
    }
    red[tid] = acc;
    block_partial_and_finish(F, R, red);
}

// true residual r = b - q (q = M x in FP64); (r, r) -> FIN_OUTER
__global__ void __launch_bounds__(256) k_residual_rr(double* __restrict__ r, const double* __restrict__ b,
                                                    const double* __restrict__ q, int64_t n, int R, FinArgs F) {
    __shared__ double red[256];
    const int rows = 256 / R, tid = threadIdx.x, rr = tid % R, lr = tid / R;
    double acc = 0.0;
    if (lr < rows) {
        const int64_t stride = (int64_t)gridDim.x * rows;
        DotAcc<double> c[4];
        int64_t i = (int64_t)blockIdx.x * rows + lr;
        for (; i + 3 * stride < n; i += 4 * stride) {
            double bv[4], qv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = (i + u * stride) * R + rr;
                bv[u] = b[k];
                qv[u] = q[k];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double v = bv[u] - qv[u];
                r[(i + u * stride) * R + rr] = v;
                c[u].add(v, v);
            }
        }
        for (; i < n; i += stride) {
            const int64_t k = i * R + rr;
            const double v = b[k] - q[k];
            r[k] = v;
            c[0].add(v, v);
        }
        acc = (c[0].value() + c[1].value()) + (c[2].value() + c[3].value());
    }
    red[tid] = acc;
    block_partial_and_finish(F, R, red);
}

// ---- batched (segmented) variants: vectors are one rhs each of n_mesh independent systems;
// thread block s works on the dofs [seg[2s], seg[2s+1]) of mesh seg_mesh[s] and the last block
// reduces, mesh by mesh, the partials of that mesh's blocks in a fixed order (one warp per
// mesh: fixed lane assignment, fixed shuffle tree).
struct SegArgs {
    const int32_t* seg_mesh;   // [nseg] mesh of each segment
    const int64_t* seg;        // [2 * nseg] begin, end of each segment
    const int32_t* mseg;       // [M + 1] first segment of each mesh
    int M;
};

__device__ void seg_partial_and_finish(const FinArgs& F, const SegArgs& G, double* red) {
    const int tid = threadIdx.x;
    __shared__ unsigned int s_last;
    __shared__ int cnt_s[256];
    for (int h = 128; h > 0; h >>= 1) {
        __syncthreads();
        if (tid < h) red[tid] += red[tid + h];
    }
    __syncthreads();
    if (tid == 0) F.partial[blockIdx.x] = red[0];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(F.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int warp = tid / 32, lane = tid % 32;
    for (int m = warp; m < G.M; m += 8) {
        const int g0 = G.mseg[m], g1 = G.mseg[m + 1];
        double v = 0.0;
        for (int g = g0 + lane; g < g1; g += 32) v += __ldcg(&F.partial[g]);
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) apply_fin(F, G.M, m, v);
    }
    __syncthreads();
    int c = 0;
    for (int m = tid; m < G.M; m += 256) c += F.flags[m];
    cnt_s[tid] = c;
    for (int h = 128; h > 0; h >>= 1) {
        __syncthreads();
        if (tid < h) cnt_s[tid] += cnt_s[tid + h];
    }
    __syncthreads();
    if (tid == 0) {
        fin_tail(F, G.M, cnt_s[0]);
        *F.ticket = 0u;
    }
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_seg_dot(const TA* __restrict__ a, const TB* __restrict__ b, SegArgs G,
                                                 FinArgs F) {
    __shared__ double red[256];
    using TD = typename DotType<TA, TB>::type;
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    DotAcc<TD> acc;
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) acc.add((TD)a[i], (TD)b[i]);
    red[threadIdx.x] = acc.value();
    seg_partial_and_finish(F, G, red);
}

template <typename T>
__global__ void __launch_bounds__(256) k_seg_update_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                       const T* __restrict__ q, const double* __restrict__ alpha,
                                                       SegArgs G, FinArgs F) {
    __shared__ double red[256];
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    const T a = (T)alpha[G.seg_mesh[blockIdx.x]];
    DotAcc<T> acc;
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) {
        x[i] = fma(a, p[i], x[i]);
        const T v = fma(-a, q[i], r[i]);
        r[i] = v;
        acc.add(v, v);
    }
    red[threadIdx.x] = acc.value();
    seg_partial_and_finish(F, G, red);
}

__global__ void __launch_bounds__(256) k_seg_outer_init(double* __restrict__ x, double* __restrict__ r,
                                                       const double* __restrict__ b, SegArgs G, FinArgs F) {
    __shared__ double red[256];
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    DotAcc<double> acc;
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) {
        const double v = b[i];
        r[i] = v;
        x[i] = 0.0;
        acc.add(v, v);
    }
    red[threadIdx.x] = acc.value();
    seg_partial_and_finish(F, G, red);
}

__global__ void __launch_bounds__(256) k_seg_inner_start(const double* __restrict__ r, const double* __restrict__ s,
                                                        float* __restrict__ r32, float* __restrict__ x32,
                                                        float* __restrict__ p32, SegArgs G, FinArgs F) {
    __shared__ double red[256];
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    const double sc = s[G.seg_mesh[blockIdx.x]];
    DotAcc<float> acc;
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) {
        const float v = (float)(r[i] * sc);
        r32[i] = v;
        x32[i] = 0.f;
        p32[i] = 0.f;
        acc.add(v, v);
    }
    red[threadIdx.x] = acc.value();
    seg_partial_and_finish(F, G, red);
}

__global__ void __launch_bounds__(256) k_seg_residual_rr(double* __restrict__ r, const double* __restrict__ b,
                                                        const double* __restrict__ q, SegArgs G, FinArgs F) {
    __shared__ double red[256];
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    DotAcc<double> acc;
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) {
        const double v = b[i] - q[i];
        r[i] = v;
        acc.add(v, v);
    }
    red[threadIdx.x] = acc.value();
    seg_partial_and_finish(F, G, red);
}

template <typename T>
__global__ void k_seg_update_p(T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ beta, SegArgs G) {
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    const T bt = (T)beta[G.seg_mesh[blockIdx.x]];
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) p[i] = fma(bt, p[i], z[i]);
}

// x += d * f with f = ||r|| (the inverse of the scale that made the inner right-hand side;
// 0 for a slot that is not refined)
__global__ void k_seg_accum_f32(double* __restrict__ x, const float* __restrict__ d, const double* __restrict__ f,
                                SegArgs G) {
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    const double sc = f[G.seg_mesh[blockIdx.x]];
    if (!(sc > 0.0)) return;
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) x[i] = fma((double)d[i], sc, x[i]);
}

// p = beta p + z.  One right-hand side with 16-byte aligned vectors (vec): 16-byte accesses,
// four in flight per array and thread, the same arithmetic per element.
template <typename T>
__global__ void k_update_p(T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ beta, int64_t nv, int R,
                           int vec) {
    pdl_launch();
    pdl_wait();
    if (vec) {
        using V = typename Vec4<T>::type;
        constexpr int W = Vec4<T>::W;
        V* pv = reinterpret_cast<V*>(p);
        const V* zv = reinterpret_cast<const V*>(z);
        const T b = (T)beta[0];
        const int64_t nvec = nv / W, stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        int64_t i = gid;
        for (; i + 3 * stride < nvec; i += 4 * stride) {
            V a[4], c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = pv[i + u * stride];
                c[u] = zv[i + u * stride];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int j = 0; j < W; ++j) vget(a[u], j) = fma(b, vget(a[u], j), vget(c[u], j));
                pv[i + u * stride] = a[u];
            }
        }
        for (; i < nvec; i += stride) {
            V a = pv[i];
            V c = zv[i];
#pragma unroll
            for (int j = 0; j < W; ++j) vget(a, j) = fma(b, vget(a, j), vget(c, j));
            pv[i] = a;
        }
        if (gid < nv - nvec * W) p[nvec * W + gid] = fma(b, p[nvec * W + gid], z[nvec * W + gid]);
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma((T)beta[R == 1 ? 0 : i % R], p[i], z[i]);
}

template <typename T>
__global__ void k_jacobi(const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ diag, int64_t nv, int R) {
    pdl_launch();
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] / diag[R == 1 ? i : i / R];
}

// x64 += (double)d32 * f_r  (f_r = ||r||: undoes the scaling of the inner right-hand side)
__global__ void k_accum_f32(double* __restrict__ x, const float* __restrict__ d, const double* __restrict__ f,
                            int64_t nv, int R) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double sr = f[R == 1 ? 0 : i % R];
        if (sr > 0.0) x[i] = fma((double)d[i], sr, x[i]);
    }
}
// Chebyshev direction update d = c1[k] d + c2[k] z, k = iterations done (read on the device,
// so that one captured body serves every iteration); coefficients [2][kmax + 1][S].
__global__ void k_update_d(double* __restrict__ d, const double* __restrict__ z, const double* __restrict__ coef,
                           const int* __restrict__ iparam, int kmax, int64_t nv, int R) {
    const int k = min(iparam[1], kmax);
    const double* c1 = coef + (size_t)k * R;
    const double* c2 = coef + (size_t)(kmax + 1 + k) * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = R == 1 ? 0 : (int)(i % R);
        d[i] = fma(c1[r], d[i], c2[r] * z[i]);
    }
}
template <typename SA>
__global__ void k_seg_update_d(double* __restrict__ d, const double* __restrict__ z, const double* __restrict__ coef,
                               const int* __restrict__ iparam, int kmax, SA G) {
    const int k = min(iparam[1], kmax);
    const int m = G.seg_mesh[blockIdx.x];
    const double a = coef[(size_t)k * G.M + m], b = coef[(size_t)(kmax + 1 + k) * G.M + m];
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) d[i] = fma(a, d[i], b * z[i]);
}

// Power iteration: v = z / sqrt(s) per rhs (or per mesh)
__global__ void k_scale_cols(double* __restrict__ v, const double* __restrict__ z, const double* __restrict__ s,
                             int64_t nv, int R) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double sr = s[R == 1 ? 0 : i % R];
        v[i] = sr > 0.0 ? z[i] / sqrt(sr) : 0.0;
    }
}
template <typename SA>
__global__ void k_seg_scale_cols(double* __restrict__ v, const double* __restrict__ z, const double* __restrict__ s,
                                 SA G) {
    const double sr = s[G.seg_mesh[blockIdx.x]];
    const double f = sr > 0.0 ? 1.0 / sqrt(sr) : 0.0;
    const int64_t beg = G.seg[2 * blockIdx.x], end = G.seg[2 * blockIdx.x + 1];
    for (int64_t i = beg + threadIdx.x; i < end; i += 256) v[i] = z[i] * f;
}

// ---- host helpers ------------------------------------------------------------------------
static int grid_for(int64_t nv) { return (int)std::max<int64_t>(1, std::min<int64_t>((nv + 255) / 256, 148 * 8)); }

static FinArgs fin_args(PcgWork* w, int kind, int* iparam = nullptr, cudaGraphConditionalHandle cond = 0,
                        bool in_graph = false) {
    FinArgs F;
    F.in_graph = in_graph ? 1 : 0;
    F.hist = w->hist;
    F.hist_cap = w->hist_cap;
    F.kind = kind;
    F.partial = w->partial;
    F.ticket = w->ticket;
    F.sc = w->sc;
    F.flags = w->flags;
    F.dparam = w->dparam;
    F.iparam = iparam;
    F.cond = cond;
    return F;
}

static SegArgs seg_args(const bras_ctx* c) {
    SegArgs G;
    G.seg_mesh = c->seg_mesh;
    G.seg = c->seg_beg;
    G.mseg = c->mseg;
    G.M = c->n_mesh;
    return G;
}

static bool batched(const bras_ctx* c) { return c->n_mesh > 1 && c->nseg > 0; }
static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Blocks of 256 threads of `kern` that the device keeps resident at once (all SMs), cached per
// (kernel, device).
static int resident_blocks(const void* kern) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kern, dev);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess) cudaGetLastError();
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int v = std::max(1, per_sm) * std::max(1, sms);
    cache[key] = v;
    return v;
}

// Blocks of a fused reduction over n x R values: about 4,096 values a block (16 per thread),
// a multiple of the 148 SMs, between 148 and one wave of resident blocks (at most
// kDotBlocks): the grid-stride loops then run in a single wave, without a partial second one.
// A function of the context's size, R and the kernel only, so every call of a context sums in
// the same order (bit-reproducible); small systems get short reduction tails.
static int dot_blocks(const bras_ctx* c, int R, const void* kern) {
    const int64_t want = (c->n * (int64_t)R + 4095) / 4096;
    const int64_t b = (want + 147) / 148 * 148;
    const int64_t cap = std::min<int64_t>(kDotBlocks, resident_blocks(kern));
    return (int)std::max<int64_t>(std::min<int64_t>(148, cap), std::min<int64_t>(cap, b));
}

// Dot products / fused updates on either layout: R interleaved rhs, or (batched) one rhs per
// mesh with n_mesh scalar slots.
template <typename TA, typename TB>
static cudaError_t vdot(bras_ctx* c, const TA* a, const TB* b, int R, int kind, cudaStream_t st) {
    PcgWork* w = c->pcg;
    if (batched(c)) k_seg_dot<TA, TB><<<c->nseg, 256, 0, st>>>(a, b, seg_args(c), fin_args(w, kind));
    else {
        const int vec = (R == 1 && std::is_same<TA, TB>::value && aligned16(a) && aligned16(b)) ? 1 : 0;
        const cudaError_t e = launch_pdl(k_dot<TA, TB>, dim3(dot_blocks(c, R, (const void*)k_dot<TA, TB>)), dim3(256), 0,
                                         st, a, b, c->n, R, vec, fin_args(w, kind));
        if (e != cudaSuccess) return e;
    }
    count_launch(1);
    return cudaGetLastError();
}

// x += alpha p; r -= alpha q; (r, r) -> `kind` (FIN_RR for CG, FIN_RR_STAT for the stationary
// iterations).  Iterations are counted on the device (iparam[IP_DONE]); inside a solve graph
// the count and the active slots set the loop condition (Chebyshev also indexes its
// coefficients by the count).
template <typename T>
static cudaError_t vupdate_xr(bras_ctx* c, T* x, T* r, const T* p, const T* q, int R, cudaGraphConditionalHandle cond,
                              cudaStream_t st, bool in_graph, int kind = FIN_RR) {
    PcgWork* w = c->pcg;
    const int S = batched(c) ? c->n_mesh : R;
    int* ip = w->iparam;
    if (batched(c))
        k_seg_update_xr<T><<<c->nseg, 256, 0, st>>>(x, r, p, q, w->sc + S_ALPHA * S, seg_args(c),
                                                     fin_args(w, kind, ip, cond, in_graph));
    else {
        const cudaError_t e = launch_pdl(
            k_update_xr<T>, dim3(dot_blocks(c, R, (const void*)k_update_xr<T>)), dim3(256), 0, st, x, r, p, q,
            (const double*)(w->sc + S_ALPHA * S), c->n, R,
            (R == 1 && aligned16(x) && aligned16(r) && aligned16(p) && aligned16(q)) ? 1 : 0,
            fin_args(w, kind, ip, cond, in_graph));
        if (e != cudaSuccess) return e;
    }
    count_launch(1);
    return cudaGetLastError();
}

static cudaError_t vupdate_d(bras_ctx* c, double* d, const double* z, int R, cudaStream_t st) {
    PcgWork* w = c->pcg;
    if (batched(c))
        k_seg_update_d<SegArgs><<<c->nseg, 256, 0, st>>>(d, z, w->coef, w->iparam, w->coef_k, seg_args(c));
    else
        k_update_d<<<grid_for(c->n * R), 256, 0, st>>>(d, z, w->coef, w->iparam, w->coef_k, c->n * R, R);
    count_launch(1);
    return cudaGetLastError();
}

static cudaError_t vscale_cols(bras_ctx* c, double* v, const double* z, int R, cudaStream_t st) {
    PcgWork* w = c->pcg;
    const int S = batched(c) ? c->n_mesh : R;
    if (batched(c))
        k_seg_scale_cols<SegArgs><<<c->nseg, 256, 0, st>>>(v, z, w->sc + S_RR * S, seg_args(c));
    else
        k_scale_cols<<<grid_for(c->n * R), 256, 0, st>>>(v, z, w->sc + S_RR * S, c->n * R, R);
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t vupdate_p(bras_ctx* c, T* p, const T* z, int R, cudaStream_t st) {
    PcgWork* w = c->pcg;
    const int S = batched(c) ? c->n_mesh : R;
    if (batched(c)) k_seg_update_p<T><<<c->nseg, 256, 0, st>>>(p, z, w->sc + S_BETA * S, seg_args(c));
    else {
        const int vec = (R == 1 && aligned16(p) && aligned16(z)) ? 1 : 0;
        const cudaError_t e = launch_pdl(k_update_p<T>, dim3(grid_for(c->n * R)), dim3(256), 0, st, p, z,
                                         (const double*)(w->sc + S_BETA * S), c->n * R, R, vec);
        if (e != cudaSuccess) return e;
    }
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t jacobi_launch(const bras_ctx* c, int prec, const void* x, void* y, int nrhs, cudaStream_t st) {
    const int64_t nv = c->n * nrhs;
    const cudaError_t e =
        prec == BRAS_FP64
            ? launch_pdl(k_jacobi<double>, dim3(grid_for(nv)), dim3(256), 0, st, (const double*)x, (double*)y,
                         (const double*)c->diag64, nv, nrhs)
            : launch_pdl(k_jacobi<float>, dim3(grid_for(nv)), dim3(256), 0, st, (const float*)x, (float*)y,
                         (const float*)c->diag32, nv, nrhs);
    count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
static int precond(bras_ctx* c, int pc, int prec, const T* r, T* z, int R, cudaStream_t st) {
    if (pc == BRAS_PC_BRAS) return run_op(c, prec, OP_BRAS, r, z, R, st);
    if (pc == BRAS_PC_JACOBI) return jacobi_launch(c, prec, r, z, R, st) == cudaSuccess ? BRAS_OK : BRAS_ERR_CUDA;
    return cudaMemcpyAsync(z, r, sizeof(T) * c->n * R, cudaMemcpyDeviceToDevice, st) == cudaSuccess ? BRAS_OK
                                                                                                   : BRAS_ERR_CUDA;
}

#define CK(x)                                   \
    do {                                        \
        if ((x) != cudaSuccess) return BRAS_ERR_CUDA; \
    } while (0)
#define RC(x)                         \
    do {                              \
        int _rc = (x);                \
        if (_rc != BRAS_OK) return _rc; \
    } while (0)

// One CG iteration (the body of the device-side while loop), enqueued on `st`:
//   z = Pr; beta = (r,z)/(r,z)_old (0 on the first pass); p = z + beta p;
//   q = M p; alpha = (r,z)/(p,q); x += alpha p; r -= alpha q; (r,r) -> convergence masks,
// and the loop condition (some rhs still active and fewer than maxit iterations).
template <typename T>
static int enqueue_iteration(bras_ctx* c, int prec, int pc, T* x, T* r, T* z, T* p, T* q, int R,
                             cudaGraphConditionalHandle cond, cudaStream_t st, bool in_graph = true) {
    PcgWork* w = c->pcg;
    const int64_t n = c->n, nv = n * R;
    RC(precond(c, pc, prec, r, z, R, st));
    CK(vdot(c, r, z, R, FIN_BETA, st));
    CK(vupdate_p<T>(c, p, z, R, st));
    RC(run_op(c, prec, OP_MASS, p, q, R, st));
    CK(vdot(c, p, q, R, FIN_ALPHA, st));
    CK(vupdate_xr<T>(c, x, r, p, q, R, cond, st, in_graph));
    (void)w;
    (void)n;
    (void)nv;
    return BRAS_OK;
}

// One iteration of a stationary method (FP64), enqueued on `st`:
//   fixed point (Sec. 3):  z = Mt^{-1} r;  q = M z;  x += w z;  r -= w q
//   Chebyshev (Sec. 3):    z = Mt^{-1} r;  d = c1[k] d + c2[k] z;  q = M d;  x += d;  r -= q
// w = omega (1 for Chebyshev) while the rhs is active, 0 once it has converged; (r, r) gives
// the stopping test and the loop condition, as in CG.  r is the recurrence residual.
static int enqueue_stationary(bras_ctx* c, int solver, int pc, double* x, double* r, double* z, double* d, double* q,
                              int R, cudaGraphConditionalHandle cond, cudaStream_t st, bool in_graph) {
    RC(precond(c, pc, BRAS_FP64, r, z, R, st));
    double* dir = z;
    if (solver == SOLVER_CHEBYSHEV) {
        CK(vupdate_d(c, d, z, R, st));
        dir = d;
    }
    RC(run_op(c, BRAS_FP64, OP_MASS, dir, q, R, st));
    CK(vupdate_xr<double>(c, x, r, dir, q, R, cond, st, in_graph, FIN_RR_STAT));
    return BRAS_OK;
}

// The whole CG loop as one graph: a conditional WHILE node (default value 1 at every launch)
// whose body is one iteration; the residual-check kernel sets the condition on the device,
// so a solve costs one graph launch and one host synchronisation.  Graphs are cached per
// (precision, preconditioner, nrhs, value type, buffers) and rebuilt if buffers change.
template <typename T>
static int get_graph(bras_ctx* c, int prec, int pc, int R, T* x, T* r, T* z, T* p, T* q, cudaGraphExec_t* out,
                     int* kernels_per_iter, int solver = SOLVER_CG) {
    PcgWork* w = c->pcg;
    for (auto& g : w->graphs)
        if (g.solver == solver && g.prec == prec && g.pc == pc && g.R == R && g.tsize == (int)sizeof(T) && g.x == x &&
            g.part == c->part && (solver != SOLVER_CHEBYSHEV || (g.coef == w->coef && g.coef_k == w->coef_k))) {
            *out = g.exec;
            *kernels_per_iter = g.kernels_per_iter;
            return BRAS_OK;
        }
    SolveGraph g;
    g.solver = solver;
    g.coef = w->coef;
    g.coef_k = w->coef_k;
    g.prec = prec;
    g.pc = pc;
    g.R = R;
    g.tsize = (int)sizeof(T);
    g.x = x;
    g.part = c->part;
    CK(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(w->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const int64_t before = launches_so_far();
    int rc = BRAS_ERR_INVALID;
    if (solver == SOLVER_CG) {
        rc = enqueue_iteration<T>(c, prec, pc, x, r, z, p, q, R, cond, w->cap);
    } else if constexpr (sizeof(T) == 8) {
        rc = enqueue_stationary(c, solver, pc, reinterpret_cast<double*>(x), reinterpret_cast<double*>(r),
                                reinterpret_cast<double*>(z), reinterpret_cast<double*>(p),
                                reinterpret_cast<double*>(q), R, cond, w->cap, true);
    }
    g.kernels_per_iter = (int)(launches_so_far() - before);
    count_launch(-g.kernels_per_iter);      // captured, not launched
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(w->cap, &captured);
    if (rc != BRAS_OK || ec != cudaSuccess) {
        cudaGraphDestroy(g.graph);
        cudaGetLastError();
        return rc != BRAS_OK ? rc : BRAS_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
        cudaGraphDestroy(g.graph);
        return BRAS_ERR_CUDA;
    }
    w->graphs.push_back(g);
    *out = g.exec;
    *kernels_per_iter = g.kernels_per_iter;
    return BRAS_OK;
}

// BRAS_SOLVE_HOST_LOOP=1 in the environment runs the CG iterations from a host loop instead of
// the conditional-while graph (identical kernels; for profilers).
static bool host_loop() {
    static const bool on = [] {
        const char* e = std::getenv("BRAS_SOLVE_HOST_LOOP");
        return e && e[0] == '1';
    }();
    return on;
}

// PCG on M x = b (b on the device, type T); x starts at 0.  Per-rhs iteration counts land in
// w->flags[R..2R), squared residual norms in w->sc[S_RR], [S_RR0].
template <typename T>
static int pcg_core(bras_ctx* c, int prec, int pc, const T* b, T* x, T* r, T* z, T* p, T* q, int R, double rtol,
                    int maxit, cudaStream_t st) {
    PcgWork* w = c->pcg;
    const int64_t n = c->n, nv = n * R;
    const int S = batched(c) ? c->n_mesh : R;    // scalar slots (rhs, or meshes of a batch)
    (void)n;
    cudaGraphExec_t exec = nullptr;
    int kpi = 0;
    RC(get_graph<T>(c, prec, pc, R, x, r, z, p, q, &exec, &kpi));
    w->h_param[0] = rtol * rtol;
    int* hp = reinterpret_cast<int*>(w->h_param + 1);
    hp[0] = maxit;
    hp[1] = 0;
    CK(cudaMemcpyAsync(w->dparam, w->h_param, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->iparam, hp, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(x, 0, sizeof(T) * nv, st));
    CK(cudaMemsetAsync(p, 0, sizeof(T) * nv, st));
    CK(cudaMemcpyAsync(r, b, sizeof(T) * nv, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(w->flags + 2 * S + 1, 0, sizeof(int), st));
    CK(vdot(c, r, r, R, FIN_INIT_RR, st));
    if (maxit > 0 && host_loop()) {
        // profiling aid: the same iteration kernels launched one by one, the stopping test read
        // back after every iteration (tools that cannot look inside conditional graphs see them)
        for (int it = 0; it < maxit; ++it) {
            RC(enqueue_iteration<T>(c, prec, pc, x, r, z, p, q, R, 0, st, false));
            CK(cudaMemcpyAsync(w->h_flags, w->flags, sizeof(int) * (2 * S + 2), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (w->h_flags[2 * S] == 0 || w->h_flags[2 * S + 1] != 0) break;
        }
        kpi = 0;
    } else if (maxit > 0) {
        CK(cudaGraphLaunch(exec, st));
        count_graph_launch();
    }
    CK(cudaMemcpyAsync(w->h_flags, w->flags, sizeof(int) * (2 * S + 2), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(double) * S_COUNT * S, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp, w->iparam, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (maxit > 0) count_launch(kpi * hp[1]);
    if (w->h_flags[2 * S + 1] != 0) return w->h_flags[2 * S + 1];
    return w->h_flags[2 * S] > 0 ? BRAS_NOT_CONVERGED : BRAS_OK;
}

// ---- mixed solve: FP64 iterative refinement around an FP32 (or BF16-inverse) inner PCG ----
// Refinement step j (slot s refined while ||r_j|| / ||b|| > rtol):
//   r32 = (float)(r_j / ||r_j||);  inner PCG on M d = r32 to the tolerance
//   tin = clamp(0.5 rtol / max_s(||r_j|| / ||b||), 1e-6, 1e-2);  x += ||r_j|| d (FP64);
//   r_{j+1} = b - M x (FP64 cell products, exact dof sums); stop when every slot passes, the
// inner iterations charged (at least one per step) reach maxit, a step broke down, or after
// kMaxOuter steps.  All of it runs from device scalars: one graph launch per solve.
static cudaError_t enqueue_outer_init(bras_ctx* c, int R, cudaGraphConditionalHandle cond, cudaStream_t st,
                                      bool in_graph) {
    PcgWork* w = c->pcg;
    const int S = batched(c) ? c->n_mesh : R;
    cudaError_t e = cudaMemsetAsync(w->flags + 2 * S + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const FinArgs F = fin_args(w, FIN_OUTER_INIT, w->iparam, cond, in_graph);
    if (batched(c)) k_seg_outer_init<<<c->nseg, 256, 0, st>>>(w->xs, w->r, w->bs, seg_args(c), F);
    else k_outer_init<<<dot_blocks(c, R, (const void*)k_outer_init), 256, 0, st>>>(w->xs, w->r, w->bs, c->n, R, F);
    count_launch(1);
    return cudaGetLastError();
}

static cudaError_t enqueue_inner_start(bras_ctx* c, int R, cudaGraphConditionalHandle cond, cudaStream_t st,
                                       bool in_graph) {
    PcgWork* w = c->pcg;
    const int S = batched(c) ? c->n_mesh : R;
    const FinArgs F = fin_args(w, FIN_INIT_INNER, w->iparam, cond, in_graph);
    if (batched(c))
        k_seg_inner_start<<<c->nseg, 256, 0, st>>>(w->r, w->sc + S_SCALE * S, w->r32, w->x32, w->p32, seg_args(c), F);
    else
        k_inner_start<<<dot_blocks(c, R, (const void*)k_inner_start), 256, 0, st>>>(w->r, w->sc + S_SCALE * S, w->r32, w->x32,
                                                                              w->p32, c->n, R, F);
    count_launch(1);
    return cudaGetLastError();
}

// inner CG iteration on the FP32 buffers (q32 serves as the search direction's image M p)
static int enqueue_inner_iteration(bras_ctx* c, int inner_prec, int pc, int R, cudaGraphConditionalHandle cond,
                                   cudaStream_t st, bool in_graph) {
    PcgWork* w = c->pcg;
    return enqueue_iteration<float>(c, inner_prec, pc, w->x32, w->r32, w->z32, w->p32, w->q32, R, cond, st, in_graph);
}

// x += ||r|| d; q = M x (FP64); r = b - q; (r, r) -> FIN_OUTER
static int enqueue_outer_post(bras_ctx* c, int R, cudaGraphConditionalHandle cond, cudaStream_t st, bool in_graph) {
    PcgWork* w = c->pcg;
    const int S = batched(c) ? c->n_mesh : R;
    const int64_t nv = c->n * R;
    if (batched(c)) k_seg_accum_f32<<<c->nseg, 256, 0, st>>>(w->xs, w->x32, w->sc + S_ISCALE * S, seg_args(c));
    else k_accum_f32<<<grid_for(nv), 256, 0, st>>>(w->xs, w->x32, w->sc + S_ISCALE * S, nv, R);
    count_launch(1);
    CK(cudaGetLastError());
    RC(run_op(c, BRAS_FP64X, OP_MASS, w->xs, w->q, R, st));
    const FinArgs F = fin_args(w, FIN_OUTER, w->iparam, cond, in_graph);
    if (batched(c)) k_seg_residual_rr<<<c->nseg, 256, 0, st>>>(w->r, w->bs, w->q, seg_args(c), F);
    else k_residual_rr<<<dot_blocks(c, R, (const void*)k_residual_rr), 256, 0, st>>>(w->r, w->bs, w->q, c->n, R, F);
    count_launch(1);
    CK(cudaGetLastError());
    return BRAS_OK;
}

// Append a conditional WHILE node (handle h) to the graph that `st` is capturing into, after
// everything captured so far; later captures on `st` depend on it.  Returns its body graph.
static int capture_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return BRAS_ERR_CUDA;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = np.conditional.phGraph_out[0];
    return BRAS_OK;
}

struct MixedKernels {
    int init = 0, start = 0, iter = 0, post = 0;   // kernels launched by each part
};

// The mixed solve as one graph:  init -> WHILE(outer) { inner start -> WHILE(inner) { CG
// iteration } -> accumulate, true residual, test }.  Cached per (inner precision,
// preconditioner, nrhs, partial buffer); every vector is a workspace buffer.
static int get_mixed_graph(bras_ctx* c, int inner_prec, int pc, int R, cudaGraphExec_t* out, MixedKernels* kn) {
    PcgWork* w = c->pcg;
    for (auto& g : w->graphs)
        if (g.solver == SOLVER_MIXED && g.prec == inner_prec && g.pc == pc && g.R == R && g.x == w->xs &&
            g.part == c->part) {
            *out = g.exec;
            *kn = MixedKernels{g.mixed_init, g.mixed_start, g.kernels_per_iter, g.mixed_post};
            return BRAS_OK;
        }
    SolveGraph g;
    g.solver = SOLVER_MIXED;
    g.prec = inner_prec;
    g.pc = pc;
    g.R = R;
    g.x = w->xs;
    g.part = c->part;
    CK(cudaGraphCreate(&g.graph, 0));
    MixedKernels k;
    int rc = BRAS_OK;
    auto counted = [&](int* cnt, auto&& fn) {
        const int64_t before = launches_so_far();
        const int r = fn();
        *cnt = (int)(launches_so_far() - before);
        count_launch(-*cnt);     // captured, not launched
        return r;
    };
    auto fail = [&](int r) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(w->cap, &junk);
        cudaGraphDestroy(g.graph);
        cudaGetLastError();
        return r;
    };
    cudaGraphConditionalHandle h_outer, h_inner;
    CK(cudaGraphConditionalHandleCreate(&h_outer, g.graph, 0, cudaGraphCondAssignDefault));
    // top level: init, then the outer loop
    CK(cudaStreamBeginCaptureToGraph(w->cap, g.graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaGraph_t outer_body = nullptr, inner_body = nullptr;
    rc = counted(&k.init, [&] { return enqueue_outer_init(c, R, h_outer, w->cap, true) == cudaSuccess ? BRAS_OK : BRAS_ERR_CUDA; });
    if (rc == BRAS_OK) rc = capture_while(w->cap, h_outer, &outer_body);
    if (rc != BRAS_OK) return fail(rc);
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(w->cap, &captured) != cudaSuccess) return fail(BRAS_ERR_CUDA);
    // outer body: inner start, the inner loop, accumulate + true residual + test
    if (cudaGraphConditionalHandleCreate(&h_inner, outer_body, 0, 0) != cudaSuccess ||
        cudaStreamBeginCaptureToGraph(w->cap, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess) {
        cudaGraphDestroy(g.graph);
        return BRAS_ERR_CUDA;
    }
    rc = counted(&k.start, [&] { return enqueue_inner_start(c, R, h_inner, w->cap, true) == cudaSuccess ? BRAS_OK : BRAS_ERR_CUDA; });
    if (rc == BRAS_OK) rc = capture_while(w->cap, h_inner, &inner_body);
    if (rc == BRAS_OK) rc = counted(&k.post, [&] { return enqueue_outer_post(c, R, h_outer, w->cap, true); });
    if (rc != BRAS_OK) return fail(rc);
    if (cudaStreamEndCapture(w->cap, &captured) != cudaSuccess) return fail(BRAS_ERR_CUDA);
    // inner body: one CG iteration
    if (cudaStreamBeginCaptureToGraph(w->cap, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess) {
        cudaGraphDestroy(g.graph);
        return BRAS_ERR_CUDA;
    }
    rc = counted(&k.iter, [&] { return enqueue_inner_iteration(c, inner_prec, pc, R, h_inner, w->cap, true); });
    if (rc != BRAS_OK) return fail(rc);
    if (cudaStreamEndCapture(w->cap, &captured) != cudaSuccess) return fail(BRAS_ERR_CUDA);
    if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
        cudaGraphDestroy(g.graph);
        cudaGetLastError();
        return BRAS_ERR_CUDA;
    }
    g.mixed_init = k.init;
    g.mixed_start = k.start;
    g.kernels_per_iter = k.iter;
    g.mixed_post = k.post;
    w->graphs.push_back(g);
    *out = g.exec;
    *kn = k;
    return BRAS_OK;
}

static bool host_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

int pcg_solve_impl(bras_ctx* c, int pc, int mode, int inner_prec, const double* b, double* x, int R, double rtol,
                   int maxit, int* iters, double* relres, cudaStream_t st) {
    if (R > kMaxRhs) return BRAS_ERR_TOO_LARGE;
    if (batched(c) && R != 1) return BRAS_ERR_INVALID;
    const int S = batched(c) ? c->n_mesh : R;     // scalar slots: rhs, or meshes of a batch
    const bool mixed = mode == BRAS_SOLVE_MIXED;
    RC(ensure_pcg(c, R, mixed));
    RC(ensure_part(c, R));
    PcgWork* w = c->pcg;
    const int64_t n = c->n, nv = n * R;
    const bool hb = host_ptr(b), hx = host_ptr(x);
    const double* db = b;
    double* dx = x;
    if (hb) {
        CK(cudaMemcpyAsync(w->bs, b, sizeof(double) * nv, cudaMemcpyHostToDevice, st));
        db = w->bs;
    }
    if (hx) dx = w->xs;
    int status = BRAS_OK;
    std::vector<int> its(S, 0);
    std::vector<double> rel(S, 0.0);
    if (!mixed) {
        status = pcg_core<double>(c, BRAS_FP64, pc, db, w->xs, w->r, w->z, w->p, w->q, R, rtol, maxit, st);
        if (status < 0) return status;
        if (dx != w->xs) CK(cudaMemcpyAsync(dx, w->xs, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        for (int r = 0; r < S; ++r) {
            its[r] = w->h_flags[S + r];
            const double rr0 = w->h_sc[S_RR0 * S + r];
            rel[r] = rr0 > 0 ? std::sqrt(w->h_sc[S_RR * S + r] / rr0) : 0.0;
        }
    } else {
        // the whole refinement loop is one graph on workspace buffers: b -> bs, result from xs
        if (!hb && b != w->bs) CK(cudaMemcpyAsync(w->bs, b, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        cudaGraphExec_t exec = nullptr;
        MixedKernels kn;
        RC(get_mixed_graph(c, inner_prec, pc, R, &exec, &kn));
        w->h_param[1] = rtol;
        int* hp = reinterpret_cast<int*>(w->h_param + 2);
        for (int k = 0; k < IP_COUNT; ++k) hp[k] = 0;
        hp[IP_MAXIT_ALL] = std::max(maxit, 0);
        CK(cudaMemcpyAsync(w->dparam + 1, w->h_param + 1, sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(w->iparam, hp, sizeof(int) * IP_COUNT, cudaMemcpyHostToDevice, st));
        if (host_loop()) {
            // profiling aid: the graph's kernels launched one by one, each loop condition read back
            auto go = [&](int which) -> int {
                if (cudaMemcpyAsync(hp, w->iparam, sizeof(int) * IP_COUNT, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return -1;
                return hp[which];
            };
            CK(enqueue_outer_init(c, R, 0, st, false));
            int g_out;
            while ((g_out = go(IP_GO_OUTER)) == 1) {
                CK(enqueue_inner_start(c, R, 0, st, false));
                int g_in;
                while ((g_in = go(IP_GO_INNER)) == 1) RC(enqueue_inner_iteration(c, inner_prec, pc, R, 0, st, false));
                if (g_in < 0) return BRAS_ERR_CUDA;
                RC(enqueue_outer_post(c, R, 0, st, false));
            }
            if (g_out < 0) return BRAS_ERR_CUDA;
        } else {
            CK(cudaGraphLaunch(exec, st));
            count_graph_launch();
        }
        CK(cudaMemcpyAsync(w->h_flags, w->flags, sizeof(int) * (3 * S + 2), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(double) * S_COUNT * S, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hp, w->iparam, sizeof(int) * IP_COUNT, cudaMemcpyDeviceToHost, st));
        if (dx != w->xs) CK(cudaMemcpyAsync(dx, w->xs, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
        if (!host_loop())
            count_launch(kn.init + (int64_t)hp[IP_OUTER] * (kn.start + kn.post) + (int64_t)hp[IP_DONE_ALL] * kn.iter);
        bool ok = true;
        for (int r = 0; r < S; ++r) {
            const double bn = w->h_sc[S_BN * S + r];
            its[r] = w->h_flags[2 * S + 2 + r];
            rel[r] = bn > 0 ? w->h_sc[S_RN * S + r] / bn : 0.0;
            if (!(rel[r] <= rtol)) ok = false;
        }
        if (w->h_flags[2 * S + 1] != 0) return w->h_flags[2 * S + 1];
        status = ok ? BRAS_OK : BRAS_NOT_CONVERGED;
    }
    if (hx) CK(cudaMemcpyAsync(x, dx, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int r = 0; r < S; ++r) {
        if (iters) iters[r] = its[r];
        if (relres) relres[r] = rel[r];
    }
    return status;
}

// Damped fixed point or Chebyshev semi-iteration in FP64 (Sec. 3).  step[s] = omega (fixed
// point) per scalar slot; lo[s], hi[s] = the spectral interval (Chebyshev).
int stationary_solve_impl(bras_ctx* c, int solver, int pc, const double* step, const double* lo, const double* hi,
                          const double* b, double* x, int R, double rtol, int maxit, int* iters, double* relres,
                          cudaStream_t st) {
    if (R > kMaxRhs) return BRAS_ERR_TOO_LARGE;
    if (batched(c) && R != 1) return BRAS_ERR_INVALID;
    const int S = batched(c) ? c->n_mesh : R;
    RC(ensure_pcg(c, R, false));
    RC(ensure_part(c, R));
    PcgWork* w = c->pcg;
    const int64_t nv = c->n * R;
    std::vector<double> scale(S, 1.0);
    if (solver == SOLVER_FIXED_POINT)
        for (int s = 0; s < S; ++s) scale[s] = step[s];
    if (solver == SOLVER_CHEBYSHEV) {
        // direction coefficients, data independent: c1[0] = 0, c2[0] = 1/theta; for k >= 1
        // rho_k = 1 / (2 sigma - rho_{k-1}) (rho_0 = 1/sigma), c1[k] = rho_k rho_{k-1}, c2[k] = 2 rho_k / delta
        const int K = std::max(maxit, 1);
        if (w->coef_k < K) {
            dfree(c, w->coef);
            w->coef = (double*)dalloc_bytes(c, sizeof(double) * 2 * (size_t)(K + 1) * w->slots);
            if (!w->coef) { w->coef_k = 0; return BRAS_ERR_OOM; }
            w->coef_k = K;
        }
        const int KM = w->coef_k;
        std::vector<double> cf(2 * (size_t)(KM + 1) * S, 0.0);
        for (int s = 0; s < S; ++s) {
            const double theta = 0.5 * (hi[s] + lo[s]), delta = 0.5 * (hi[s] - lo[s]), sigma = theta / delta;
            cf[(size_t)(KM + 1) * S + s] = 1.0 / theta;
            double rho = 1.0 / sigma;
            for (int k = 1; k <= KM; ++k) {
                const double rn = 1.0 / (2.0 * sigma - rho);
                cf[(size_t)k * S + s] = rn * rho;
                cf[(size_t)(KM + 1 + k) * S + s] = 2.0 * rn / delta;
                rho = rn;
            }
        }
        // slot stride S: the update kernels index [k][S]
        CK(cudaMemcpyAsync(w->coef, cf.data(), sizeof(double) * cf.size(), cudaMemcpyHostToDevice, st));
    }
    const bool hb = host_ptr(b), hx = host_ptr(x);
    const double* db = b;
    if (hb) {
        CK(cudaMemcpyAsync(w->bs, b, sizeof(double) * nv, cudaMemcpyHostToDevice, st));
        db = w->bs;
    }
    cudaGraphExec_t exec = nullptr;
    int kpi = 0;
    RC(get_graph<double>(c, BRAS_FP64, pc, R, w->xs, w->r, w->z, w->p, w->q, &exec, &kpi, solver));
    w->h_param[0] = rtol * rtol;
    int* hp = reinterpret_cast<int*>(w->h_param + 1);
    hp[0] = maxit;
    hp[1] = 0;
    CK(cudaMemcpyAsync(w->dparam, w->h_param, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->iparam, hp, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->sc + S_SCALE * S, scale.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w->xs, 0, sizeof(double) * nv, st));
    CK(cudaMemsetAsync(w->p, 0, sizeof(double) * nv, st));
    CK(cudaMemcpyAsync(w->r, db, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(w->flags + 2 * S + 1, 0, sizeof(int), st));
    CK(vdot(c, w->r, w->r, R, FIN_INIT_STAT, st));
    if (maxit > 0 && host_loop()) {
        for (int it = 0; it < maxit; ++it) {
            RC(enqueue_stationary(c, solver, pc, w->xs, w->r, w->z, w->p, w->q, R, 0, st, false));
            CK(cudaMemcpyAsync(w->h_flags, w->flags, sizeof(int) * (2 * S + 2), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (w->h_flags[2 * S] == 0 || w->h_flags[2 * S + 1] != 0) break;
        }
        kpi = 0;
    } else if (maxit > 0) {
        CK(cudaGraphLaunch(exec, st));
        count_graph_launch();
    }
    if (hx) CK(cudaMemcpyAsync(x, w->xs, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
    else if (x != w->xs) CK(cudaMemcpyAsync(x, w->xs, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(w->h_flags, w->flags, sizeof(int) * (2 * S + 2), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(double) * S_COUNT * S, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp, w->iparam, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (maxit > 0 && kpi > 0) count_launch(kpi * hp[1]);
    for (int s = 0; s < S; ++s) {
        const double rr0 = w->h_sc[S_RR0 * S + s];
        if (iters) iters[s] = w->h_flags[S + s];
        if (relres) relres[s] = rr0 > 0 ? std::sqrt(w->h_sc[S_RR * S + s] / rr0) : 0.0;
    }
    if (w->h_flags[2 * S + 1] != 0) return w->h_flags[2 * S + 1];
    return w->h_flags[2 * S] > 0 ? BRAS_NOT_CONVERGED : BRAS_OK;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm sequence of the
// LDL^T pivots).
static int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        const double off = i ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// CG-Lanczos: `steps` FP64 PCG iterations on M x = b record alpha_k, beta_k; the tridiagonal
// T[j][j] = 1/alpha_j + beta_j/alpha_{j-1}, T[j][j+1] = sqrt(beta_{j+1})/alpha_j of the Lanczos
// process on Mt^{-1} M has extreme eigenvalues (found by bisection) that approach
// lambda_min, lambda_max of Mt^{-1} M from inside.
int cg_lanczos_impl(bras_ctx* c, int pc, const double* b, int steps, double* lmin, double* lmax, int* done,
                    cudaStream_t st) {
    if (batched(c)) return BRAS_ERR_INVALID;
    RC(ensure_pcg(c, 1, false));
    RC(ensure_part(c, 1));
    PcgWork* w = c->pcg;
    const int64_t n = c->n;
    double* hist = (double*)dalloc_bytes(c, sizeof(double) * 2 * (size_t)steps);
    if (!hist) return BRAS_ERR_OOM;
    CK(cudaMemsetAsync(hist, 0, sizeof(double) * 2 * (size_t)steps, st));
    CK(cudaMemcpyAsync(w->r, b, sizeof(double) * n, host_ptr(b) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(w->xs, 0, sizeof(double) * n, st));
    CK(cudaMemsetAsync(w->p, 0, sizeof(double) * n, st));
    w->h_param[0] = 1e-28;   // stop below 1e-14 ||b||: beyond it the coefficients carry only rounding
    int* hp = reinterpret_cast<int*>(w->h_param + 1);
    hp[0] = steps;
    hp[1] = 0;
    CK(cudaMemcpyAsync(w->dparam, w->h_param, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->iparam, hp, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w->flags + 3, 0, sizeof(int), st));
    w->hist = hist;
    w->hist_cap = steps;
    int rc = BRAS_OK;
    if (vdot(c, w->r, w->r, 1, FIN_INIT_RR, st) != cudaSuccess) rc = BRAS_ERR_CUDA;
    for (int it = 0; it < steps && rc == BRAS_OK; ++it)
        rc = enqueue_iteration<double>(c, BRAS_FP64, pc, w->xs, w->r, w->z, w->p, w->q, 1, 0, st, false);
    w->hist = nullptr;     // solve graphs never see the history buffer
    w->hist_cap = 0;
    std::vector<double> h(2 * (size_t)steps);
    if (rc == BRAS_OK &&
        (cudaMemcpyAsync(w->h_flags, w->flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaMemcpyAsync(h.data(), hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        rc = BRAS_ERR_CUDA;
    dfree(c, hist);
    if (rc != BRAS_OK) return rc;
    if (w->h_flags[3] != 0) return w->h_flags[3];
    const int k = std::min(steps, w->h_flags[1]);   // iterations done
    if (done) *done = k;
    if (k < 1) return BRAS_ERR_BREAKDOWN;
    std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
    for (int j = 0; j < k; ++j) {
        d[j] = 1.0 / h[j] + (j ? h[steps + j] / h[j - 1] : 0.0);
        if (j + 1 < k) e[j] = std::sqrt(h[steps + j + 1]) / h[j];
    }
    double lo = d[0], hi = d[0];   // Gershgorin bracket
    for (int j = 0; j < k; ++j) {
        const double rad = (j ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < k ? std::fabs(e[j]) : 0.0);
        lo = std::min(lo, d[j] - rad);
        hi = std::max(hi, d[j] + rad);
    }
    auto bisect = [&](int index) {   // the eigenvalue with `index` eigenvalues below it
        double a = lo, bb = hi;
        for (int it = 0; it < 200 && bb - a > 1e-15 * std::max(std::fabs(a), std::fabs(bb)); ++it) {
            const double m = 0.5 * (a + bb);
            if (sturm_count(d, e, m) <= index) a = m;
            else bb = m;
        }
        return 0.5 * (a + bb);
    };
    *lmin = bisect(0);
    *lmax = bisect(k - 1);
    return BRAS_OK;
}

// lambda_max of Mt^{-1} M by the power iteration (Sec. 3): w = M v; z = Mt^{-1} w;
// lambda = (w, z) / (w, v) (the Rayleigh quotient in the M inner product); v = z / ||z||.
int lambda_max_impl(bras_ctx* c, int pc, const double* v0, int R, int iters, double* lambda, cudaStream_t st) {
    if (R > kMaxRhs) return BRAS_ERR_TOO_LARGE;
    if (batched(c) && R != 1) return BRAS_ERR_INVALID;
    const int S = batched(c) ? c->n_mesh : R;
    RC(ensure_pcg(c, R, false));
    RC(ensure_part(c, R));
    PcgWork* w = c->pcg;
    const int64_t nv = c->n * R;
    CK(cudaMemcpyAsync(w->xs, v0, sizeof(double) * nv, host_ptr(v0) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < iters; ++it) {
        RC(run_op(c, BRAS_FP64, OP_MASS, w->xs, w->q, R, st));
        RC(precond(c, pc, BRAS_FP64, w->q, w->z, R, st));
        CK(vdot(c, w->q, w->z, R, FIN_STORE_A, st));
        CK(vdot(c, w->q, w->xs, R, FIN_STORE_B, st));
        CK(vdot(c, w->z, w->z, R, FIN_NORM, st));
        CK(vscale_cols(c, w->xs, w->z, R, st));
    }
    CK(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(double) * S_COUNT * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int s = 0; s < S; ++s) {
        const double den = w->h_sc[S_PQ * S + s];
        lambda[s] = den > 0 ? w->h_sc[S_RZ * S + s] / den : 0.0;
    }
    return BRAS_OK;
}

}  // namespace bras
