// extern "C" entry points of libbras: setup, applies, solve, gradient, info, teardown.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "dispatch.h"
#include "internal.h"
#include "packet.h"
#include "refelem.h"
#include "setup_dev.h"

namespace bras {

thread_local int64_t g_detail = -1;
static std::atomic<int64_t> g_launches{0};
static std::atomic<int64_t> g_graph_launches{0};

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void count_graph_launch() { g_graph_launches.fetch_add(1, std::memory_order_relaxed); }

void set_detail(int64_t d) { g_detail = d; }

void* dalloc_bytes(bras_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    c->owned.push_back(p);
    return p;
}

void dfree(bras_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->owned.begin(), c->owned.end(), p);
    if (it != c->owned.end()) c->owned.erase(it);
    cudaFree(p);
}

namespace {

template <typename T>
T* dalloc(bras_ctx* c, size_t count) {
    return static_cast<T*>(dalloc_bytes(c, count * sizeof(T)));
}

template <typename T>
int upload(bras_ctx* c, T** dst, const T* src, size_t count) {
    *dst = dalloc<T>(c, count);
    if (!*dst) return BRAS_ERR_OOM;
    if (count && cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return BRAS_ERR_CUDA;
    return BRAS_OK;
}

template <typename T>
int fetch(std::vector<T>& dst, const T* src, size_t count) {
    dst.resize(count);
    if (count && cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDefault) != cudaSuccess) return BRAS_ERR_CUDA;
    return BRAS_OK;
}

// Cholesky inverse of an SPD matrix in long double (the H1 reference mass, once per setup).
bool spd_inverse(const std::vector<double>& M, int n, std::vector<double>& inv) {
    std::vector<long double> L((size_t)n * n, 0);
    for (int j = 0; j < n; ++j) {
        long double s = M[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0)) return false;
        L[(size_t)j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            long double t = M[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / L[(size_t)j * n + j];
        }
    }
    std::vector<long double> W((size_t)n * n, 0);   // W = L^{-1}
    for (int c = 0; c < n; ++c) {
        W[(size_t)c * n + c] = 1 / L[(size_t)c * n + c];
        for (int i = c + 1; i < n; ++i) {
            long double s = 0;
            for (int k = c; k < i; ++k) s += L[(size_t)i * n + k] * W[(size_t)k * n + c];
            W[(size_t)i * n + c] = -s / L[(size_t)i * n + i];
        }
    }
    inv.assign((size_t)n * n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            long double s = 0;
            for (int k = std::max(i, j); k < n; ++k) s += W[(size_t)k * n + i] * W[(size_t)k * n + j];
            inv[(size_t)i * n + j] = (double)s;
        }
    return true;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

cudaError_t to_float(const double* a, float* b, int64_t n, cudaStream_t st) {
    int nb = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
    if (nb < 1) nb = 1;
    k_to_float<<<nb, 256, 0, st>>>(a, b, n);
    count_launch(1);
    return cudaGetLastError();
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Replace the context's block tables (cell order, multiplicities and per-cell data do not
// depend on the block size, so only these change).
int install_tables(bras_ctx* c, const HostTables& t) {
    for (void* p : {(void*)c->blk_e0, (void*)c->blk_u0, (void*)c->blk_nint, (void*)c->blk_p0, (void*)c->blk_pkt,
                    (void*)c->pkt, (void*)c->sh_items, (void*)c->sh_d, (void*)c->grp_rec, (void*)c->grp_slots})
        if (p) dfree(c, p);
    c->blk_e0 = c->blk_u0 = c->blk_nint = c->blk_p0 = nullptr;
    c->sh_items = nullptr;
    c->sh_d = nullptr;
    c->grp_rec = nullptr;
    c->grp_slots = nullptr;
    c->blk_pkt = nullptr;
    c->pkt = nullptr;
    c->BE = t.BE;
    c->nblk = t.nblk;
    c->max_u = t.max_u;
    c->max_ne = t.max_ne;
    c->U_tot = t.U_tot;
    c->npart = t.npart;
    c->nsh = t.nsh;
    {   // at most 2^h copies of a dof in a block.  FP32 / bf16: parts of L = min(22, 30 - h)
        // bits (|ql| <= 2^(L-1): sums below 2^29), products below 2^fx_top with fx_top =
        // min(L + 21, 31 + L - h) (|qh| < 2^21 for the FP32 rounding, high sums below 2^31).
        // Float-float mass: low words of 31 - h bits, fx_top = 60 - 2h.  FP64: 61 - h.
        int h = 0;
        while ((1 << h) < t.max_copies) ++h;
        if (h > 20) return BRAS_ERR_TOO_LARGE;
        c->fx_lo = std::min(22, 30 - h);
        c->fx_top = std::min(c->fx_lo + 21, 31 + c->fx_lo - h);
        c->fx_lo_df = 31 - h;
        c->fx_top_df = 60 - 2 * h;
        c->fx_top64 = 61 - h;
    }
    c->ngrp = (int64_t)t.grp_size.size();
    c->max_pkt = t.max_pkt;
    int rc;
    if ((rc = upload(c, &c->blk_e0, t.blk_e0.data(), t.blk_e0.size()))) return rc;
    if ((rc = upload(c, &c->blk_u0, t.blk_u0.data(), t.blk_u0.size()))) return rc;
    if ((rc = upload(c, &c->blk_nint, t.blk_nint.data(), t.blk_nint.size()))) return rc;
    if ((rc = upload(c, &c->blk_p0, t.blk_p0.data(), t.blk_p0.size()))) return rc;
    if ((rc = upload(c, &c->blk_pkt, t.blk_pkt.data(), t.blk_pkt.size()))) return rc;
    if ((rc = upload(c, &c->pkt, t.pkt.data(), t.pkt.size()))) return rc;
    {   // the combine pass's records: items (dof, group) in group order, groups (first item,
        // block count, first slot entry)
        const size_t ng = t.grp_size.size();
        std::vector<int2> items(t.sh_ids.size());
        std::vector<int4> rec(ng);
        for (size_t g = 0; g < ng; ++g) {
            rec[g] = make_int4(t.grp_item0[g], t.grp_cnt[g], t.grp_slot0[g], 0);
            for (int32_t j = t.grp_item0[g]; j < t.grp_item0[g + 1]; ++j) items[j] = make_int2(t.sh_ids[j], (int)g);
        }
        if ((rc = upload(c, &c->sh_items, items.data(), items.size()))) return rc;
        if ((rc = upload(c, &c->grp_rec, rec.data(), rec.size()))) return rc;
    }
    if ((rc = upload(c, &c->grp_slots, t.grp_slots.data(), t.grp_slots.size()))) return rc;
    if ((rc = upload(c, &c->sh_d, t.sh_d.data(), t.sh_d.size()))) return rc;
    return BRAS_OK;
}

int setup_impl(bras_ctx* c, int dim, int space, int order, int64_t n_vert, const double* coords,
               int64_t n_cell, const int32_t* cells, int64_t n_dof, const int32_t* l2g, const int8_t* signs,
               const double* rho, const bras_options* opt, cudaStream_t st, const int32_t* cell_group = nullptr) {
    const int basis = opt ? opt->basis : 0;
    if (basis < 0 || basis > 2) return BRAS_ERR_INVALID;   // n_local rejects the pairs that do not exist
    const int nloc = n_local(dim, space, order, basis);
    c->dim = dim;
    c->space = space;
    c->order = order;
    c->nloc = nloc;
    c->ncomp = space == BRAS_H1 ? 1 : 3;
    c->E = n_cell;
    c->n = n_dof;
    c->nvert = n_vert;
    c->precisions = (opt && opt->precisions) ? opt->precisions : 7;
    c->max_nrhs = (opt && opt->max_nrhs > 0) ? opt->max_nrhs : 1;
    int BE = (opt && opt->block_elems) ? opt->block_elems : 256;
    // H1 contexts on the FP32 units (no tensor-core kernel) take blocks of up to 1024 cells,
    // the block kernels looping over the cells of a block; the others up to 256
    const bool simt_h1 = space == BRAS_H1 && !(h1_tc_supported(nloc) && !(opt && opt->simt_only));
    if (BE < 32 || BE > (simt_h1 ? 1024 : 256)) return BRAS_ERR_INVALID;
    c->BE = BE;
    const bool want64 = c->precisions & 1, want32 = c->precisions & 2, wantbf = c->precisions & 4;

    // host copies (inputs may live on either side)
    std::vector<double> h_coords;
    std::vector<int32_t> h_cells, h_l2g;
    std::vector<int8_t> h_signs;
    int rc;
    if ((rc = fetch(h_coords, coords, (size_t)n_vert * dim))) return rc;
    if ((rc = fetch(h_cells, cells, (size_t)n_cell * (dim + 1)))) return rc;
    if ((rc = fetch(h_l2g, l2g, (size_t)n_cell * nloc))) return rc;
    if (signs && (rc = fetch(h_signs, signs, (size_t)n_cell * nloc))) return rc;
    for (size_t i = 0; i < h_cells.size(); ++i)
        if (h_cells[i] < 0 || h_cells[i] >= n_vert) { set_detail((int64_t)i); return BRAS_ERR_INVALID; }
    for (size_t i = 0; i < h_signs.size(); ++i)
        if (h_signs[i] != 1 && h_signs[i] != -1) { set_detail((int64_t)i); return BRAS_ERR_INVALID; }
    // Lagrange (H1) dofs are point values with no orientation: every sign must be +1
    if (space == BRAS_H1)
        for (size_t i = 0; i < h_signs.size(); ++i)
            if (h_signs[i] != 1) { set_detail((int64_t)i); return BRAS_ERR_INVALID; }

    // Block size: the largest multiple of 32 (<= BE) whose FP64 kernel fits the device's
    // shared memory and, unless the caller fixed it, whose FP32 kernel fits twice per SM.
    int smem_optin = 0, smem_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const bool fixed_be = opt && opt->block_elems;
    const bool want_tc = space == BRAS_H1 && h1_tc_supported(nloc) && !(opt && opt->simt_only);
    HostTables t;
    int64_t detail = -1;
    for (;;) {
        rc = build_tables(h_l2g.data(), signs ? h_signs.data() : nullptr, n_cell, nloc, n_dof, h_coords.data(),
                          h_cells.data(), dim, BE, &t, &detail, cell_group, space != BRAS_H1);
        if (rc) { set_detail(detail); return rc; }
        const size_t s64 = block_smem_estimate(nloc, 8, space == BRAS_H1, t);
        size_t s32 = block_smem_estimate(nloc, 4, space == BRAS_H1, t);
        // the FP32 tensor-core kernel: B tiles instead of the SIMT reference copy
        if (want_tc) s32 = std::max(s32, h1_tc_smem_bytes(nloc, shape_args(t)));
        // a context for several right-hand sides also wants its multi-RHS kernel (16-byte
        // chunks of every dof's row) to fit one CTA
        const size_t smr = mr_smem_estimate(c, nloc, space == BRAS_H1, want_tc, t);
        const bool fits = s64 <= (size_t)smem_optin &&
                          (fixed_be || (2 * (s32 + 1024) <= (size_t)smem_sm && smr <= (size_t)smem_optin));
        if (fits || BE <= 32) {
            if (s64 > (size_t)smem_optin) return BRAS_ERR_TOO_LARGE;
            break;
        }
        BE = std::max(32, (BE - 32) & ~31);
    }
    t.BE = BE;
    if ((rc = upload(c, &c->perm, t.perm.data(), t.perm.size()))) return rc;
    if ((rc = install_tables(c, t))) return rc;
    if (!(c->status = dalloc<int>(c, 1))) return BRAS_ERR_OOM;
    if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) return BRAS_ERR_CUDA;
    if ((rc = upload(c, &c->dinv64, t.dinv.data(), t.dinv.size()))) return rc;
    if (!(c->dinv32 = dalloc<float>(c, n_dof))) return BRAS_ERR_OOM;
    if (to_float(c->dinv64, c->dinv32, n_dof, st) != cudaSuccess) return BRAS_ERR_CUDA;

    // many right-hand sides on streamed cell matrices: the cells' maps in internal order with
    // P's sign in bit 31, and the dof-sorted slots of the copies (ascending (cell, local index))
    if (space != BRAS_H1 && nloc <= kCellMrMaxLoc && c->max_nrhs >= kCellMrMinRhs) {
        const size_t m = (size_t)n_cell * nloc;
        std::vector<int32_t> ml(m), slot(m);
        std::vector<int64_t> off((size_t)n_dof + 1, 0);
        for (int64_t e = 0; e < n_cell; ++e) {
            const int64_t K = t.perm[e];
            for (int a = 0; a < nloc; ++a) {
                const int32_t g = h_l2g[(size_t)K * nloc + a];
                const bool neg = signs && h_signs[(size_t)K * nloc + a] < 0;
                ml[(size_t)e * nloc + a] = neg ? (int32_t)((uint32_t)g | 0x80000000u) : g;
                off[(size_t)g + 1]++;
            }
        }
        for (int64_t u = 0; u < n_dof; ++u) off[u + 1] += off[u];
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (size_t i = 0; i < m; ++i) slot[i] = (int32_t)fill[ml[i] & 0x7fffffff]++;
        if ((rc = upload(c, &c->mr_l2g, ml.data(), m))) return rc;
        if ((rc = upload(c, &c->mr_slot, slot.data(), m))) return rc;
        if ((rc = upload(c, &c->mr_off, off.data(), off.size()))) return rc;
    }

    // reference tables (library construction, host)
    RefTables ref;
    if (build_reference(dim, space, order, &ref, basis) != 0) return BRAS_ERR_INVALID;

    // mixed Poisson Schur complement tables (RT on tetrahedra): divergence block, the caller's
    // l2g with P's signs times sign(det J_K), and the dof-sorted order of the broken copies
    if (space == BRAS_HDIV && dim == 3 && ref.nq > 0) {
        c->nq = ref.nq;
        std::vector<float> b32(ref.Bdiv.begin(), ref.Bdiv.end());
        if ((rc = upload(c, &c->Bdiv64, ref.Bdiv.data(), ref.Bdiv.size()))) return rc;
        if ((rc = upload(c, &c->Bdiv32, b32.data(), b32.size()))) return rc;
        std::vector<int8_t> sg((size_t)n_cell * nloc);
        for (int64_t K = 0; K < n_cell; ++K) {
            const double* x0 = &h_coords[(size_t)h_cells[K * 4] * 3];
            double J[3][3];
            for (int j = 0; j < 3; ++j)
                for (int r = 0; r < 3; ++r) J[r][j] = h_coords[(size_t)h_cells[K * 4 + j + 1] * 3 + r] - x0[r];
            const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            for (int a = 0; a < nloc; ++a)
                sg[(size_t)K * nloc + a] = (int8_t)((signs ? h_signs[(size_t)K * nloc + a] : 1) * (det < 0 ? -1 : 1));
        }
        std::vector<int64_t> off((size_t)n_dof + 1, 0);
        for (size_t i = 0; i < h_l2g.size(); ++i) off[(size_t)h_l2g[i] + 1]++;
        for (int64_t i = 0; i < n_dof; ++i) off[i + 1] += off[i];
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        std::vector<int32_t> pos(h_l2g.size());
        for (size_t i = 0; i < h_l2g.size(); ++i) pos[i] = (int32_t)fill[h_l2g[i]]++;
        if ((rc = upload(c, &c->l2g_user, h_l2g.data(), h_l2g.size()))) return rc;
        if ((rc = upload(c, &c->sgn_user, sg.data(), sg.size()))) return rc;
        if ((rc = upload(c, &c->cpos, pos.data(), pos.size()))) return rc;
        if ((rc = upload(c, &c->coff, off.data(), off.size()))) return rc;
    }

    // device copies of the geometry inputs
    const double* d_coords = coords;
    const int32_t* d_cells = cells;
    const double* d_rho = rho;
    if (!is_device_ptr(coords)) {
        double* p;
        if ((rc = upload(c, &p, h_coords.data(), h_coords.size()))) return rc;
        d_coords = p;
    }
    if (!is_device_ptr(cells)) {
        int32_t* p;
        if ((rc = upload(c, &p, h_cells.data(), h_cells.size()))) return rc;
        d_cells = p;
    }
    if (rho && !is_device_ptr(rho)) {
        std::vector<double> h_rho(rho, rho + n_cell);
        double* p;
        if ((rc = upload(c, &p, h_rho.data(), h_rho.size()))) return rc;
        d_rho = p;
    }

    unsigned long long* bad = dalloc<unsigned long long>(c, 1);
    int* nfixed = dalloc<int>(c, 1);
    if (!bad || !nfixed) return BRAS_ERR_OOM;
    const unsigned long long none = ~0ull;
    cudaMemcpy(bad, &none, sizeof(none), cudaMemcpyHostToDevice);
    cudaMemset(nfixed, 0, sizeof(int));

    if (!(c->absdet = dalloc<double>(c, n_cell)) || !(c->rho = dalloc<double>(c, n_cell))) return BRAS_ERR_OOM;
    const bool h1 = space == BRAS_H1;
    if (h1) {
        const int n = nloc;
        std::vector<double> inv;
        if (!spd_inverse(ref.R, n, inv)) return BRAS_ERR_NOT_SPD;
        // exponent bounds of the row abs-sums of M_ref and M_ref^{-1}, plus one for the rounding
        // of the FP32 / TF32 copies
        auto row_exp = [n](const std::vector<double>& A) {
            double best = 0.0;
            for (int r = 0; r < n; ++r) {
                double s = 0.0;
                for (int q = 0; q < n; ++q) s += std::fabs(A[(size_t)r * n + q]);
                best = std::max(best, s);
            }
            int ex = 0;
            std::frexp(best, &ex);
            return ex + 1;
        };
        c->er_mass = row_exp(ref.R);
        c->er_bras = row_exp(inv);
        std::vector<float> R32(ref.R.begin(), ref.R.end()), I32(inv.begin(), inv.end());
        if ((rc = upload(c, &c->Mref64, ref.R.data(), ref.R.size()))) return rc;
        if ((rc = upload(c, &c->Minvref64, inv.data(), inv.size()))) return rc;
        if ((rc = upload(c, &c->Mref32, R32.data(), R32.size()))) return rc;
        if ((rc = upload(c, &c->Minvref32, I32.data(), I32.size()))) return rc;
        if (want_tc) {
            std::vector<unsigned char> tm, ti;
            h1_tc_build_btile(ref.R.data(), n, tm);
            h1_tc_build_btile(inv.data(), n, ti);
            if ((rc = upload(c, &c->btile_mass, tm.data(), tm.size()))) return rc;
            if ((rc = upload(c, &c->btile_bras, ti.data(), ti.size()))) return rc;
            c->use_tc = true;
        }
        if (!(c->mscale64 = dalloc<double>(c, n_cell)) || !(c->bscale64 = dalloc<double>(c, n_cell)) ||
            !(c->mscale32 = dalloc<float>(c, n_cell)) || !(c->bscale32 = dalloc<float>(c, n_cell)))
            return BRAS_ERR_OOM;
    } else {
        if (!(c->metric = dalloc<double>(c, (size_t)6 * n_cell))) return BRAS_ERR_OOM;
        if ((rc = upload(c, &c->Rref, ref.R.data(), ref.R.size()))) return rc;
    }
    if (run_geometry(dim, space, n_cell, c->perm, d_coords, d_cells, d_rho, c->absdet, c->rho, c->metric,
                     c->mscale64, c->bscale64, c->mscale32, c->bscale32, bad, st) != cudaSuccess)
        return BRAS_ERR_CUDA;
    unsigned long long hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BRAS_ERR_CUDA;
    if (hbad != none) { set_detail((int64_t)hbad); return BRAS_ERR_DEGENERATE; }

    if (!h1) {
        c->npk = nloc * (nloc + 1) / 2;
        c->Epad = (n_cell + 31) / 32 * 32;
        const size_t cnt = (size_t)pk_groups(c->npk, 8) * 8 * c->Epad;   // whole 16-byte groups
        // FP64 tables are always built (outer residual, diag); FP32 / bf16 on request
        // FP64 cell matrices always (refinement residual, diag); FP64 inverses only when the FP64
        // precision is asked for (the FP64 BRAS apply)
        if (!(c->Mpk64 = dalloc<double>(c, cnt))) return BRAS_ERR_OOM;
        if (want64 && !(c->Minvpk64 = dalloc<double>(c, cnt))) return BRAS_ERR_OOM;
        if (want32 || wantbf) {
            if (!(c->Mpk32 = dalloc<float>(c, cnt))) return BRAS_ERR_OOM;
        }
        if (want32 && !(c->Minvpk32 = dalloc<float>(c, cnt))) return BRAS_ERR_OOM;
        if (wantbf && !(c->Minvpkbf = dalloc<__nv_bfloat16>(c, cnt))) return BRAS_ERR_OOM;
        // zero the padding entries of the last 16-byte groups
        if (cudaMemsetAsync(c->Mpk64, 0, cnt * 8, st) != cudaSuccess ||
            (c->Minvpk64 && cudaMemsetAsync(c->Minvpk64, 0, cnt * 8, st) != cudaSuccess) ||
            (c->Mpk32 && cudaMemsetAsync(c->Mpk32, 0, cnt * 4, st) != cudaSuccess) ||
            (c->Minvpk32 && cudaMemsetAsync(c->Minvpk32, 0, cnt * 4, st) != cudaSuccess) ||
            (c->Minvpkbf && cudaMemsetAsync(c->Minvpkbf, 0, cnt * 2, st) != cudaSuccess))
            return BRAS_ERR_CUDA;
        if (run_element_inverse(nloc, n_cell, c->Epad, c->Rref, c->metric, c->Mpk64, c->Mpk32, c->Minvpk64,
                                c->Minvpk32, c->Minvpkbf, bad, nfixed, c->perm, st) != cudaSuccess)
            return BRAS_ERR_CUDA;
        if (cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&c->bf16_fixed, nfixed, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return BRAS_ERR_CUDA;
        if (hbad != none) { set_detail((int64_t)hbad); return BRAS_ERR_NOT_SPD; }
        // many right-hand sides: the FP64 cell matrices as float pairs for the float-float
        // refinement residual
        if (c->mr_l2g) {
            if (!(c->Mpkdf = dalloc<float2>(c, cnt))) return BRAS_ERR_OOM;
            if (run_split_pairs(c->Mpk64, c->Mpkdf, cnt, st) != cudaSuccess) return BRAS_ERR_CUDA;
        }
        // exponent bounds of the cells' row abs-sums (plus one for the FP32 / bf16 roundings)
        int* eb = dalloc<int>(c, 2);
        if (!eb) return BRAS_ERR_OOM;
        const int lo[2] = {-100000, -100000};
        int he[2] = {0, 0};
        if (cudaMemcpy(eb, lo, sizeof(lo), cudaMemcpyHostToDevice) != cudaSuccess ||
            run_row_bound(nloc, n_cell, c->Epad, c->Mpk64, eb, st) != cudaSuccess ||
            (c->Minvpk64 ? run_row_bound(nloc, n_cell, c->Epad, c->Minvpk64, eb + 1, st)
                         : c->Minvpk32 ? run_row_bound(nloc, n_cell, c->Epad, c->Minvpk32, eb + 1, st)
                                       : run_row_bound(nloc, n_cell, c->Epad, c->Minvpkbf, eb + 1, st)) != cudaSuccess ||
            cudaMemcpyAsync(he, eb, sizeof(he), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return BRAS_ERR_CUDA;
        c->er_mass = he[0] + 1;
        c->er_bras = he[1] + 1;
    }

    // Block-size autotuner (opt-in): time the FP32 (else FP64) BRAS apply with the block tables
    // of every admissible size -- multiples of 32 up to 256 whose FP64 and FP32 / tensor-core
    // kernels fit the opt-in shared memory -- and keep the fastest.
    if (ensure_part(c, c->max_nrhs) != BRAS_OK) return BRAS_ERR_OOM;
    if (opt && opt->autotune && !fixed_be) {
        const int prec = has_precision(c, BRAS_FP32) ? BRAS_FP32 : BRAS_FP64;
        const size_t w = prec == BRAS_FP64 ? 8 : 4;
        void* xv = dalloc_bytes(c, w * (size_t)n_dof);
        void* yv = dalloc_bytes(c, w * (size_t)n_dof);
        if (!xv || !yv) return BRAS_ERR_OOM;
        {   // a fixed pseudo-random input (the timing does not depend on the values)
            std::vector<double> hx((size_t)n_dof);
            uint64_t z = 0x9E3779B97F4A7C15ull;
            for (auto& v : hx) {
                z ^= z << 13;
                z ^= z >> 7;
                z ^= z << 17;
                v = (double)(z >> 11) * 0x1.0p-53 - 0.5;
            }
            if (prec == BRAS_FP64) {
                if (cudaMemcpy(xv, hx.data(), 8 * hx.size(), cudaMemcpyHostToDevice) != cudaSuccess) return BRAS_ERR_CUDA;
            } else {
                std::vector<float> hf(hx.begin(), hx.end());
                if (cudaMemcpy(xv, hf.data(), 4 * hf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return BRAS_ERR_CUDA;
            }
        }
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BRAS_ERR_CUDA;
        HostTables best;
        float best_us = 1e30f;
        c->tune_count = 0;
        // candidates: larger blocks for H1 on the FP32 units (fewer shared dofs), finer steps
        // around the tensor-core kernel's two-threads-per-cell limit of 128 cells
        static const int kSimtH1[8] = {1024, 768, 512, 384, 256, 192, 128, 64};
        static const int kTc[8] = {256, 192, 160, 128, 112, 96, 80, 64};
        static const int kOther[8] = {256, 224, 192, 160, 128, 96, 64, 32};
        const int* cand = simt_h1 ? kSimtH1 : (c->use_tc ? kTc : kOther);
        for (int ci = 0; ci < 8; ++ci) {
            const int be = cand[ci];
            HostTables tt;
            if ((rc = build_tables(h_l2g.data(), signs ? h_signs.data() : nullptr, n_cell, nloc, n_dof, h_coords.data(),
                                   h_cells.data(), dim, be, &tt, &detail, cell_group, space != BRAS_H1)))
                break;
            tt.BE = be;
            const size_t s64 = block_smem_estimate(nloc, 8, space == BRAS_H1, tt);
            size_t s32 = block_smem_estimate(nloc, 4, space == BRAS_H1, tt);
            if (c->use_tc) s32 = std::max(s32, h1_tc_smem_bytes(nloc, shape_args(tt)));
            if (s64 > (size_t)smem_optin || s32 > (size_t)smem_optin) continue;
            const size_t smr = mr_smem_estimate(c, nloc, space == BRAS_H1, c->use_tc, tt);
            if (smr > (size_t)smem_optin && be > 32) continue;   // keep the multi-RHS kernel usable
            if ((rc = install_tables(c, tt)) || (rc = ensure_part(c, c->max_nrhs))) break;
            // two warm-up applies, then the mean of ten (candidates within a few percent of
            // each other need that many to be told apart)
            constexpr int kWarm = 2, kReps = 10;
            float ms = 0.f;
            bool okr = true;
            for (int r = 0; r < kWarm && okr; ++r) okr = run_op(c, prec, OP_BRAS, xv, yv, 1, st) == BRAS_OK;
            cudaEventRecord(e0, st);
            for (int r = 0; r < kReps && okr; ++r) okr = run_op(c, prec, OP_BRAS, xv, yv, 1, st) == BRAS_OK;
            cudaEventRecord(e1, st);
            if (!okr || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = BRAS_ERR_CUDA;
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            const float us = 1e3f * ms / kReps;
            if (c->tune_count < (int)(sizeof(c->tune_be) / sizeof(c->tune_be[0]))) {
                c->tune_be[c->tune_count] = be;
                c->tune_us[c->tune_count] = us;
                c->tune_count++;
            }
            if (us < best_us) {
                best_us = us;
                best = std::move(tt);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dfree(c, xv);
        dfree(c, yv);
        if (rc) return rc;
        if (best_us < 1e30f) {
            if ((rc = install_tables(c, best)) || (rc = ensure_part(c, c->max_nrhs))) return rc;
        }
    }

    // diag(M) (Jacobi, Sec. 2.1) through the same deterministic scatter as the final tables
    if (!(c->diag64 = dalloc<double>(c, n_dof)) || !(c->diag32 = dalloc<float>(c, n_dof))) return BRAS_ERR_OOM;
    if (run_op(c, BRAS_FP64, OP_DIAG, nullptr, c->diag64, 1, st) != BRAS_OK) return BRAS_ERR_CUDA;
    if (to_float(c->diag64, c->diag32, n_dof, st) != cudaSuccess) return BRAS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return BRAS_ERR_CUDA;
    return BRAS_OK;
}

}  // namespace

BlockArgs shape_args(const HostTables& t) {
    BlockArgs A{};
    A.max_pkt = t.max_pkt;
    A.max_u = t.max_u;
    A.max_ne = t.max_ne;
    return A;
}

size_t block_smem_estimate(int nloc, int tsize, bool h1, const HostTables& t, int cw) {
    const int w = tsize == 4 ? 4 : 2;
    const size_t npad = (size_t)((nloc + w - 1) / w * w);
    const size_t xsb = (size_t)tsize * (((size_t)t.max_u * cw + 3) / 4 * 4);
    if (h1)   // staged x, fixed-point accumulators, reference matrix
        return 128 + ((t.max_pkt + 127u) & ~127u) + xsb + 8 * (((size_t)t.max_u * cw + 1) / 2 * 2) +
               (size_t)tsize * nloc * npad;
    // staged x, dof-sorted products
    return 128 + ((t.max_pkt + 127u) & ~127u) + xsb + (size_t)tsize * (((size_t)nloc * t.max_ne * cw + 3) / 4 * 4);
}

// Shared memory of the FP32 multi-RHS block kernel (16-byte chunks: 4 values a dof), 0 for a
// context built for one right-hand side.
size_t mr_smem_estimate(const bras_ctx* c, int nloc, bool h1, bool tc, const HostTables& t) {
    if (c->max_nrhs <= 1) return 0;
    size_t s = block_smem_estimate(nloc, 4, h1, t, 4);
    if (tc) s = std::max(s, h1_tc_smem_bytes(nloc, shape_args(t), true));
    return s;
}

int smem_per_sm_bytes() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cached[dev] = v;
    }
    return cached[dev];
}

int smem_optin_bytes() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cached[dev] = v;
    }
    return cached[dev];
}

// Scratch entries (times element size) one apply of nrhs right-hand sides needs: the partial
// sums of shared dofs, or, on the many-right-hand-side streamed path, every copy's row.
size_t part_entries(const bras_ctx* c, int nrhs) {
    const int64_t rows = (c->mr_l2g && nrhs >= kCellMrMinRhs) ? std::max<int64_t>(c->npart, c->E * c->nloc) : c->npart;
    return (size_t)std::max<int64_t>(rows, 1) * (size_t)nrhs;
}

int ensure_part(bras_ctx* c, int nrhs) {
    size_t need = part_entries(c, nrhs) * sizeof(double);
    if (need <= c->part_bytes) return BRAS_OK;
    dfree(c, c->part);
    c->part = dalloc_bytes(c, need);
    if (!c->part) { c->part_bytes = 0; return BRAS_ERR_OOM; }
    c->part_bytes = need;
    return BRAS_OK;
}

LaunchCommon make_launch(const bras_ctx* c, int prec, int op) {
    // FP64 kernels accumulate in one 64-bit word per dof; FP32, bf16 and the H1 float-float mass
    // apply (BRAS_FP64X) in two 32-bit words, with their own splits
    const bool df = prec == BRAS_FP64X && c->space == BRAS_H1 && op == OP_MASS;
    const bool pk_df = prec == BRAS_FP64X && c->space != BRAS_H1 && op == OP_MASS;
    const bool acc64 = prec == BRAS_FP64 || (prec == BRAS_FP64X && !df);
    if (prec == BRAS_FP64X) prec = BRAS_FP64;
    LaunchCommon L{};
    BlockArgs& A = L.A;
    A.blk_e0 = c->blk_e0;
    A.blk_u0 = c->blk_u0;
    A.blk_nint = c->blk_nint;
    A.blk_p0 = c->blk_p0;
    A.blk_pkt = c->blk_pkt;
    A.pkt = c->pkt;
    A.status = c->status;
    A.Epad = c->Epad;
    A.npart = c->npart;
    A.max_u = c->max_u;
    A.max_ne = c->max_ne;
    A.max_pkt = c->max_pkt;
    A.fx_top = acc64 ? c->fx_top64 : df ? c->fx_top_df : c->fx_top;
    A.fx_lo = acc64 ? 0 : df ? c->fx_lo_df : c->fx_lo;
    A.fx_er = op == OP_BRAS ? c->er_bras : c->er_mass;
    A.mr_l2g = c->mr_l2g;
    A.mr_slot = c->mr_slot;
    A.mr_off = c->mr_off;
    A.dinv = prec == BRAS_FP64 ? (const void*)c->dinv64 : (const void*)c->dinv32;
    A.n_dof = c->n;
    A.n_cell = c->E;
    A.pk_df = pk_df ? c->Mpkdf : nullptr;
    const bool f64 = prec == BRAS_FP64;
    if (c->space == BRAS_H1) {
        if (op == OP_BRAS) {
            A.refmat = f64 ? (const void*)c->Minvref64 : (const void*)c->Minvref32;
            A.scale = f64 ? (const void*)c->bscale64 : (const void*)c->bscale32;
        } else {
            A.refmat = f64 ? (const void*)c->Mref64 : (const void*)c->Mref32;
            A.scale = f64 ? (const void*)c->mscale64 : (const void*)c->mscale32;
        }
    } else {
        if (op == OP_BRAS)
            A.pk = f64 ? (const void*)c->Minvpk64 : prec == BRAS_BF16 ? (const void*)c->Minvpkbf : (const void*)c->Minvpk32;
        else
            A.pk = f64 ? (const void*)c->Mpk64 : (const void*)c->Mpk32;
    }
    L.nblk = c->nblk;
    L.G.nsh = c->nsh;
    L.G.items = c->sh_items;
    L.G.sh_d = c->sh_d;
    L.G.grp = c->grp_rec;
    L.G.grp_slots = c->grp_slots;
    return L;
}

// The one precision / kernel dispatch of every apply; `part` holds the partial sums of the
// block-boundary dofs (npart * nrhs values of the apply's type).
int dispatch_op(const bras_ctx* c, int prec, int op, const void* x, void* y, void* part, int nrhs, cudaStream_t st) {
    LaunchCommon L = make_launch(c, prec, op);
    cudaError_t err;
    const bool h1 = c->space == BRAS_H1;
    if (prec == BRAS_FP64 || prec == BRAS_FP64X) {
        auto* xx = static_cast<const double*>(x);
        auto* yy = static_cast<double*>(y);
        auto* pp = static_cast<double*>(part);
        if (h1 && prec == BRAS_FP64X && op == OP_MASS) err = launch_h1_df(L, c->nloc, xx, yy, pp, nrhs, st);
        else err = h1 ? launch_h1_f64(L, c->nloc, op, xx, yy, pp, nrhs, st) : launch_pk_f64(L, c->nloc, op, xx, yy, pp, nrhs, st);
    } else {
        auto* xx = static_cast<const float*>(x);
        auto* yy = static_cast<float*>(y);
        auto* pp = static_cast<float*>(part);
        if (h1 && c->use_tc && (op == OP_MASS || op == OP_BRAS))
            err = launch_h1_tc(L, op == OP_MASS ? c->btile_mass : c->btile_bras, c->nloc, op, xx, yy, pp, nrhs, st);
        else if (h1) err = launch_h1_f32(L, c->nloc, op, xx, yy, pp, nrhs, st);
        else if (prec == BRAS_BF16 && op == OP_BRAS) err = launch_pk_bf16(L, c->nloc, op, xx, yy, pp, nrhs, st);
        else err = launch_pk_f32(L, c->nloc, op, xx, yy, pp, nrhs, st);
    }
    return err == cudaSuccess ? BRAS_OK : BRAS_ERR_CUDA;
}

int run_op(bras_ctx* c, int prec, int op, const void* x, void* y, int nrhs, cudaStream_t st) {
    if (ensure_part(c, nrhs) != BRAS_OK) return BRAS_ERR_OOM;
    return dispatch_op(c, prec, op, x, y, c->part, nrhs, st);
}

// FP64 BRAS apply available (H1 always; vector spaces built with the FP64 precision)
bool has_fp64_bras(const bras_ctx* c) { return c->space == BRAS_H1 || c->Minvpk64 != nullptr; }

bool has_precision(const bras_ctx* c, int prec) {
    if (prec == BRAS_FP64 || prec == BRAS_FP64X) return true;
    if (c->space == BRAS_H1) return prec == BRAS_FP32 || prec == BRAS_BF16;
    if (prec == BRAS_FP32) return c->Minvpk32 && c->Mpk32;
    if (prec == BRAS_BF16) return c->Minvpkbf && c->Mpk32;
    return false;
}

}  // namespace bras

using namespace bras;

// The context's device status word (bounded kernel waits that ran out): read after `st`
// drains; set bits turn a result `rc` into BRAS_ERR_DEVICE (detail = bits) and are cleared
// if `clear`.
static int device_status(bras_ctx* c, cudaStream_t st, int rc, bool clear) {
    int bits = 0;
    if (cudaMemcpyAsync(&bits, c->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return BRAS_ERR_CUDA;
    if (bits == 0) return rc;
    if (clear && (cudaMemsetAsync(c->status, 0, sizeof(int), st) != cudaSuccess ||
                  cudaStreamSynchronize(st) != cudaSuccess))
        return BRAS_ERR_CUDA;
    set_detail(bits);
    return BRAS_ERR_DEVICE;
}

extern "C" {

int bras_n_local(int dim, int space, int order, int basis) { return n_local(dim, space, order, basis); }

int bras_setup(bras_ctx** out, int dim, int space, int order, int64_t n_vert, const double* coords,
               int64_t n_cell, const int32_t* cells, int64_t n_dof, const int32_t* l2g, const int8_t* signs,
               const double* rho, const bras_options* opt, void* stream) {
    set_detail(-1);
    if (!out) return BRAS_ERR_INVALID;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || space < 0 || space > 2) return BRAS_ERR_INVALID;
    const int nloc = n_local(dim, space, order, opt ? opt->basis : 0);
    if (nloc < 0) return BRAS_ERR_INVALID;
    if (!coords || !cells || !l2g || n_vert <= dim || n_cell <= 0 || n_dof <= 0) return BRAS_ERR_INVALID;
    if (n_cell >= (1ll << 31) || n_dof >= (1ll << 31) || n_cell * nloc >= (1ll << 31)) return BRAS_ERR_TOO_LARGE;
    bras_ctx* c = new (std::nothrow) bras_ctx();
    if (!c) return BRAS_ERR_OOM;
    int rc = setup_impl(c, dim, space, order, n_vert, coords, n_cell, cells, n_dof, l2g, signs, rho, opt,
                        static_cast<cudaStream_t>(stream));
    if (rc != BRAS_OK) {
        bras_destroy(c);
        return rc;
    }
    *out = c;
    return BRAS_OK;
}

// Segments of at most kSegDofs dofs, each inside one mesh (the vector kernels of a batched
// solve give one thread block per segment and reduce per mesh in a fixed order).
static int build_segments(bras_ctx* c) {
    constexpr int64_t kSegDofs = 8192;
    std::vector<int32_t> smesh, mseg;
    std::vector<int64_t> sbeg;
    for (int m = 0; m < c->n_mesh; ++m) {
        mseg.push_back((int32_t)smesh.size());
        for (int64_t b = c->dof_off[m]; b < c->dof_off[m + 1]; b += kSegDofs) {
            smesh.push_back(m);
            sbeg.push_back(b);
        }
    }
    mseg.push_back((int32_t)smesh.size());
    sbeg.push_back(c->dof_off[c->n_mesh]);
    c->nseg = (int)smesh.size();
    // segment s ends at min(next start, end of its mesh)
    std::vector<int64_t> bounds(2 * (size_t)c->nseg);
    for (int s = 0; s < c->nseg; ++s) {
        bounds[2 * s] = sbeg[s];
        bounds[2 * s + 1] = std::min(sbeg[s] + kSegDofs, c->dof_off[smesh[s] + 1]);
    }
    int rc;
    if ((rc = upload(c, &c->seg_mesh, smesh.data(), smesh.size()))) return rc;
    if ((rc = upload(c, &c->seg_beg, bounds.data(), bounds.size()))) return rc;
    if ((rc = upload(c, &c->mseg, mseg.data(), mseg.size()))) return rc;
    return BRAS_OK;
}

static int apply_common(const bras_ctx* cc, int prec, int op, const void* x, void* y, int nrhs, void* stream) {
    set_detail(-1);
    if (!cc || !x || !y || nrhs < 1 || prec < 0 || prec > 3) return BRAS_ERR_INVALID;
    if (prec == BRAS_FP64X && op != OP_MASS) return BRAS_ERR_INVALID;
    if (!has_precision(cc, prec) || (prec == BRAS_FP64 && op == OP_BRAS && !has_fp64_bras(cc)))
        return BRAS_ERR_PRECISION;
    return run_op(const_cast<bras_ctx*>(cc), prec, op, x, y, nrhs, static_cast<cudaStream_t>(stream));
}

int bras_setup_batched(bras_ctx** out, int dim, int space, int order, int n_mesh, const bras_mesh_desc* meshes,
                       const bras_options* opt, void* stream) {
    set_detail(-1);
    if (!out) return BRAS_ERR_INVALID;
    *out = nullptr;
    if (!meshes || n_mesh < 1 || (dim != 2 && dim != 3) || space < 0 || space > 2) return BRAS_ERR_INVALID;
    const int nloc = n_local(dim, space, order, opt ? opt->basis : 0);
    if (nloc < 0) return BRAS_ERR_INVALID;
    int64_t V = 0, E = 0, N = 0;
    bool any_signs = false, any_rho = false;
    for (int m = 0; m < n_mesh; ++m) {
        const bras_mesh_desc& d = meshes[m];
        if (!d.coords || !d.cells || !d.l2g || d.n_vert <= dim || d.n_cell <= 0 || d.n_dof <= 0) {
            set_detail(m);
            return BRAS_ERR_INVALID;
        }
        V += d.n_vert;
        E += d.n_cell;
        N += d.n_dof;
        any_signs |= d.signs != nullptr;
        any_rho |= d.rho != nullptr;
    }
    if (E >= (1ll << 31) || N >= (1ll << 31) || E * nloc >= (1ll << 31) || V >= (1ll << 31)) return BRAS_ERR_TOO_LARGE;
    // concatenate (vertex ids and dofs shifted by the earlier meshes' counts)
    std::vector<double> coords((size_t)V * dim), rho(any_rho ? (size_t)E : 0, 1.0);
    std::vector<int32_t> cells((size_t)E * (dim + 1)), l2g((size_t)E * nloc), group((size_t)E);
    std::vector<int8_t> signs(any_signs ? (size_t)E * nloc : 0, 1);
    std::vector<int64_t> dof_off(n_mesh + 1, 0);
    int64_t v0 = 0, e0 = 0, n0 = 0;
    for (int m = 0; m < n_mesh; ++m) {
        const bras_mesh_desc& d = meshes[m];
        const size_t nc = (size_t)d.n_cell;
        if (cudaMemcpy(coords.data() + v0 * dim, d.coords, sizeof(double) * d.n_vert * dim, cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(cells.data() + e0 * (dim + 1), d.cells, sizeof(int32_t) * nc * (dim + 1), cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(l2g.data() + e0 * nloc, d.l2g, sizeof(int32_t) * nc * nloc, cudaMemcpyDefault) != cudaSuccess)
            return BRAS_ERR_CUDA;
        if (d.signs && cudaMemcpy(signs.data() + e0 * nloc, d.signs, nc * nloc, cudaMemcpyDefault) != cudaSuccess)
            return BRAS_ERR_CUDA;
        if (d.rho && cudaMemcpy(rho.data() + e0, d.rho, sizeof(double) * nc, cudaMemcpyDefault) != cudaSuccess)
            return BRAS_ERR_CUDA;
        for (size_t i = 0; i < nc * (dim + 1); ++i) {
            const int32_t vtx = cells[e0 * (dim + 1) + i];
            if (vtx < 0 || vtx >= d.n_vert) { set_detail(m); return BRAS_ERR_INVALID; }
            cells[e0 * (dim + 1) + i] = (int32_t)(vtx + v0);
        }
        for (size_t i = 0; i < nc * nloc; ++i) {
            const int32_t g = l2g[e0 * nloc + i];
            if (g < 0 || g >= d.n_dof) { set_detail(e0 * nloc + (int64_t)i); return BRAS_ERR_L2G_RANGE; }
            l2g[e0 * nloc + i] = (int32_t)(g + n0);
        }
        for (size_t k = 0; k < nc; ++k) group[e0 + k] = m;
        v0 += d.n_vert;
        e0 += d.n_cell;
        n0 += d.n_dof;
        dof_off[m + 1] = n0;
    }
    bras_ctx* c = new (std::nothrow) bras_ctx();
    if (!c) return BRAS_ERR_OOM;
    int rc = setup_impl(c, dim, space, order, V, coords.data(), E, cells.data(), N, l2g.data(),
                        any_signs ? signs.data() : nullptr, any_rho ? rho.data() : nullptr, opt,
                        static_cast<cudaStream_t>(stream), group.data());
    if (rc == BRAS_OK) {
        c->n_mesh = n_mesh;
        c->dof_off = dof_off;
        rc = build_segments(c);
    }
    if (rc != BRAS_OK) {
        bras_destroy(c);
        return rc;
    }
    *out = c;
    return BRAS_OK;
}

int bras_batch_offsets(const bras_ctx* ctx, int* n_mesh, int64_t* dof_offsets) {
    if (!ctx) return BRAS_ERR_INVALID;
    if (n_mesh) *n_mesh = ctx->n_mesh;
    if (dof_offsets) {
        if (ctx->dof_off.empty()) {
            dof_offsets[0] = 0;
            dof_offsets[1] = ctx->n;
        } else {
            for (int m = 0; m <= ctx->n_mesh; ++m) dof_offsets[m] = ctx->dof_off[m];
        }
    }
    return BRAS_OK;
}

int bras_mass_apply(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs, void* stream) {
    return apply_common(ctx, precision, OP_MASS, x, y, nrhs, stream);
}

int bras_apply(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs, void* stream) {
    return apply_common(ctx, precision, OP_BRAS, x, y, nrhs, stream);
}

int bras_jacobi_apply(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs, void* stream) {
    set_detail(-1);
    if (!ctx || !x || !y || nrhs < 1 || precision < 0 || precision > 2) return BRAS_ERR_INVALID;
    return jacobi_launch(ctx, precision, x, y, nrhs, static_cast<cudaStream_t>(stream)) == cudaSuccess ? BRAS_OK
                                                                                                        : BRAS_ERR_CUDA;
}

int bras_pcg_solve(const bras_ctx* ctx, int pc, int mode, int inner_precision, const double* b, double* x,
                   int nrhs, double rtol, int maxit, int* iters, double* relres, void* stream) {
    set_detail(-1);
    if (!ctx || !b || !x || nrhs < 1 || pc < 0 || pc > 2 || mode < 0 || mode > 1 || !(rtol >= 0) || maxit < 0)
        return BRAS_ERR_INVALID;
    if (mode == BRAS_SOLVE_MIXED && inner_precision != BRAS_FP32 && inner_precision != BRAS_BF16)
        return BRAS_ERR_INVALID;
    if (mode == BRAS_SOLVE_MIXED && !has_precision(ctx, inner_precision)) return BRAS_ERR_PRECISION;
    if (mode == BRAS_SOLVE_FP64 && pc == BRAS_PC_BRAS && !has_fp64_bras(ctx)) return BRAS_ERR_PRECISION;
    bras_ctx* c = const_cast<bras_ctx*>(ctx);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return device_status(c, st, pcg_solve_impl(c, pc, mode, inner_precision, b, x, nrhs, rtol, maxit, iters, relres, st),
                         true);
}

static int slots_of(const bras_ctx* c, int nrhs) { return (c->n_mesh > 1 && c->nseg > 0) ? c->n_mesh : nrhs; }

int bras_lambda_max(const bras_ctx* ctx, int pc, const double* v0, int nrhs, int iters, double* lambda,
                    void* stream) {
    set_detail(-1);
    if (!ctx || !v0 || !lambda || nrhs < 1 || iters < 1 || pc < 0 || pc > 2) return BRAS_ERR_INVALID;
    if (pc == BRAS_PC_BRAS && !has_fp64_bras(ctx)) return BRAS_ERR_PRECISION;
    bras_ctx* c = const_cast<bras_ctx*>(ctx);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return device_status(c, st, lambda_max_impl(c, pc, v0, nrhs, iters, lambda, st), true);
}

int bras_cg_lanczos(const bras_ctx* ctx, int pc, const double* b, int steps, double* lambda_min, double* lambda_max,
                    int* steps_done, void* stream) {
    set_detail(-1);
    if (!ctx || !b || !lambda_min || !lambda_max || steps < 1 || pc < 0 || pc > 2) return BRAS_ERR_INVALID;
    if (pc == BRAS_PC_BRAS && !has_fp64_bras(ctx)) return BRAS_ERR_PRECISION;
    bras_ctx* c = const_cast<bras_ctx*>(ctx);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return device_status(c, st, cg_lanczos_impl(c, pc, b, steps, lambda_min, lambda_max, steps_done, st), true);
}

int bras_schur_apply(const bras_ctx* ctx, int precision, const void* x, void* y, void* stream) {
    set_detail(-1);
    if (!ctx || !x || !y || (precision != BRAS_FP64 && precision != BRAS_FP32 && precision != BRAS_BF16))
        return BRAS_ERR_INVALID;
    if (ctx->nq == 0 || (ctx->n_mesh > 1 && ctx->nseg > 0)) return BRAS_ERR_INVALID;
    if (!has_precision(ctx, precision) || (precision == BRAS_FP64 && !has_fp64_bras(ctx))) return BRAS_ERR_PRECISION;
    return schur_apply_impl(const_cast<bras_ctx*>(ctx), precision, x, y, static_cast<cudaStream_t>(stream));
}

int bras_fixed_point_solve(const bras_ctx* ctx, int pc, const double* omega, const double* b, double* x, int nrhs,
                           double rtol, int maxit, int* iters, double* relres, void* stream) {
    set_detail(-1);
    if (!ctx || !omega || !b || !x || nrhs < 1 || pc < 0 || pc > 2 || !(rtol >= 0) || maxit < 0)
        return BRAS_ERR_INVALID;
    if (pc == BRAS_PC_BRAS && !has_fp64_bras(ctx)) return BRAS_ERR_PRECISION;
    const int S = slots_of(ctx, nrhs);
    for (int s = 0; s < S; ++s)
        if (!(omega[s] > 0) || !std::isfinite(omega[s])) { set_detail(s); return BRAS_ERR_INVALID; }
    bras_ctx* c = const_cast<bras_ctx*>(ctx);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return device_status(
        c, st, stationary_solve_impl(c, 1, pc, omega, nullptr, nullptr, b, x, nrhs, rtol, maxit, iters, relres, st),
        true);
}

int bras_chebyshev_solve(const bras_ctx* ctx, int pc, const double* lmin, const double* lmax, const double* b,
                         double* x, int nrhs, double rtol, int maxit, int* iters, double* relres, void* stream) {
    set_detail(-1);
    if (!ctx || !lmin || !lmax || !b || !x || nrhs < 1 || pc < 0 || pc > 2 || !(rtol >= 0) || maxit < 0)
        return BRAS_ERR_INVALID;
    if (pc == BRAS_PC_BRAS && !has_fp64_bras(ctx)) return BRAS_ERR_PRECISION;
    const int S = slots_of(ctx, nrhs);
    for (int s = 0; s < S; ++s)
        if (!(lmin[s] > 0) || !(lmax[s] > lmin[s]) || !std::isfinite(lmax[s])) { set_detail(s); return BRAS_ERR_INVALID; }
    bras_ctx* c = const_cast<bras_ctx*>(ctx);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return device_status(
        c, st, stationary_solve_impl(c, 2, pc, nullptr, lmin, lmax, b, x, nrhs, rtol, maxit, iters, relres, st),
        true);
}

int bras_grad_rho(const bras_ctx* ctx, const double* x, const double* lam, double* rho_bar, void* stream) {
    set_detail(-1);
    if (!ctx || !x || !lam || !rho_bar || ctx->space != BRAS_H1) return BRAS_ERR_INVALID;
    return grad_rho_launch(ctx, x, lam, rho_bar, false, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? BRAS_OK
               : BRAS_ERR_CUDA;
}

int bras_grad_log_rho(const bras_ctx* ctx, const double* x, const double* lam, double* z_bar, void* stream) {
    set_detail(-1);
    if (!ctx || !x || !lam || !z_bar || ctx->space != BRAS_H1) return BRAS_ERR_INVALID;
    return grad_rho_launch(ctx, x, lam, z_bar, true, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? BRAS_OK
               : BRAS_ERR_CUDA;
}

static int update_weights(bras_ctx* ctx, const double* w, bool from_log, void* stream) {
    set_detail(-1);
    if (!ctx || !w || ctx->space != BRAS_H1) return BRAS_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (update_rho_launch(ctx, w, from_log, st) != cudaSuccess) return BRAS_ERR_CUDA;
    if (run_op(ctx, BRAS_FP64, OP_DIAG, nullptr, ctx->diag64, 1, st) != BRAS_OK) return BRAS_ERR_CUDA;
    if (to_float(ctx->diag64, ctx->diag32, ctx->n, st) != cudaSuccess) return BRAS_ERR_CUDA;
    return BRAS_OK;
}

int bras_update_rho(bras_ctx* ctx, const double* rho, void* stream) { return update_weights(ctx, rho, false, stream); }

int bras_update_log_rho(bras_ctx* ctx, const double* z, void* stream) { return update_weights(ctx, z, true, stream); }

int bras_block_tuning(const bras_ctx* ctx, int* block_elems, int* count, int* sizes, float* apply_us) {
    set_detail(-1);
    if (!ctx) return BRAS_ERR_INVALID;
    if (block_elems) *block_elems = ctx->BE;
    if (count) *count = ctx->tune_count;
    for (int i = 0; i < ctx->tune_count; ++i) {
        if (sizes) sizes[i] = ctx->tune_be[i];
        if (apply_us) apply_us[i] = ctx->tune_us[i];
    }
    return BRAS_OK;
}

int bras_info(const bras_ctx* ctx, int64_t* n_dof, int64_t* n_cell, int* n_loc, int* n_blocks) {
    if (!ctx) return BRAS_ERR_INVALID;
    if (n_dof) *n_dof = ctx->n;
    if (n_cell) *n_cell = ctx->E;
    if (n_loc) *n_loc = ctx->nloc;
    if (n_blocks) *n_blocks = ctx->nblk;
    return BRAS_OK;
}

int64_t bras_algorithmic_bytes(const bras_ctx* ctx, int precision, int nrhs, int bras) {
    if (!ctx || nrhs < 1) return -1;
    const int64_t w = (precision == BRAS_FP64 || precision == BRAS_FP64X) ? 8 : 4;
    int64_t bytes = ctx->E * ctx->nloc * 4;                          // l2g map
    if (ctx->space == BRAS_H1) bytes += ctx->E * w;                  // per-cell factor
    else {
        const int64_t wi = precision == BRAS_FP64 ? 8 : (precision == BRAS_BF16 && bras ? 2 : 4);
        bytes += ctx->E * (int64_t)ctx->npk * wi;                     // packed local matrix
    }
    bytes += 2 * ctx->n * nrhs * w;                                   // x read, y written
    if (bras) bytes += ctx->n;                                        // multiplicity byte
    return bytes;
}

void bras_destroy(bras_ctx* ctx) {
    if (!ctx) return;
    free_pcg(ctx);
    for (void* p : ctx->owned) cudaFree(p);
    ctx->owned.clear();
    delete ctx;
}

const char* bras_status_string(int code) {
    switch (code) {
        case BRAS_OK: return "ok";
        case BRAS_NOT_CONVERGED: return "not converged (maxit reached)";
        case BRAS_ERR_INVALID: return "invalid argument";
        case BRAS_ERR_L2G_RANGE: return "l2g entry out of range";
        case BRAS_ERR_NO_COPY: return "dof referenced by no cell";
        case BRAS_ERR_DEGENERATE: return "degenerate cell (det J = 0) or non-positive weight";
        case BRAS_ERR_NOT_SPD: return "local mass matrix not SPD";
        case BRAS_ERR_CUDA: return "CUDA error";
        case BRAS_ERR_OOM: return "out of memory";
        case BRAS_ERR_BREAKDOWN: return "CG breakdown";
        case BRAS_ERR_PRECISION: return "precision not built in this context";
        case BRAS_ERR_TOO_LARGE: return "size above a library limit";
        case BRAS_ERR_DEVICE: return "a kernel's bounded wait ran out";
        default: return "unknown status";
    }
}

int64_t bras_last_error_detail(void) { return g_detail; }

int bras_device_status(bras_ctx* ctx, void* stream, int clear) {
    set_detail(-1);
    if (!ctx) return BRAS_ERR_INVALID;
    return device_status(ctx, static_cast<cudaStream_t>(stream), BRAS_OK, clear != 0);
}

int64_t bras_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }
int64_t bras_graph_launches(void) { return g_graph_launches.load(std::memory_order_relaxed); }

}  // extern "C"
