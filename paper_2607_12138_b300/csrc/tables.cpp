// Host construction of the deterministic scatter tables (setup time, not timed).
//
// The BRAS apply D^{-1} P^T M_br^{-1} P D^{-1} (Eq. mhatinvbras_def) and the mass apply
// P^T M_br P (Eq. M_PMbrP) both end in the transpose of the signed gather P: every conforming
// dof sums the contributions of its broken copies.  These tables let one thread block do
// that sum in on-chip memory for the dofs whose copies all live in its cells; a dof on a
// block boundary gets one partial sum per block, and the last of its blocks to finish adds
// them up in ascending block order -- no floating-point atomics.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ctx.h"
#include "packet.h"

namespace bras {
namespace {

uint64_t spread3(uint64_t v) {          // 21 bits -> every third bit
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

}  // namespace

int build_tables(const int32_t* l2g, const int8_t* signs, int64_t E, int nloc, int64_t n,
                 const double* coords, const int32_t* cells, int dim, int BE, HostTables* t,
                 int64_t* detail, const int32_t* cell_group, bool scatter) {
    // multiplicities d_i = #{(K, a) : l2g[K, a] = i}  (D = P^T P)
    std::vector<int32_t> d(n, 0);
    for (int64_t i = 0; i < E * nloc; ++i) {
        int32_t g = l2g[i];
        if (g < 0 || g >= n) { *detail = i; return BRAS_ERR_L2G_RANGE; }
        d[g]++;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (d[i] == 0) { *detail = i; return BRAS_ERR_NO_COPY; }
        if (d[i] > 65535) { *detail = i; return BRAS_ERR_TOO_LARGE; }
    }
    t->dinv.resize(n);
    for (int64_t i = 0; i < n; ++i) t->dinv[i] = 1.0 / (double)d[i];

    // Morton order of cell centroids (locality of each block's dof set)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    std::vector<double> cen((size_t)E * 3, 0.0);
    for (int64_t k = 0; k < E; ++k)
        for (int c = 0; c < dim; ++c) {
            double s = 0;
            for (int j = 0; j <= dim; ++j) s += coords[(size_t)cells[k * (dim + 1) + j] * dim + c];
            s /= (dim + 1);
            cen[k * 3 + c] = s;
            lo[c] = std::min(lo[c], s);
            hi[c] = std::max(hi[c], s);
        }
    // cells of one group (one mesh of a batch) stay contiguous: sort by (group, Morton code)
    std::vector<std::pair<std::pair<int32_t, uint64_t>, int32_t>> key(E);
    for (int64_t k = 0; k < E; ++k) {
        uint64_t code = 0;
        for (int c = 0; c < dim; ++c) {
            double span = hi[c] - lo[c];
            double f = span > 0 ? (cen[k * 3 + c] - lo[c]) / span : 0.0;
            uint64_t q = (uint64_t)std::min(2097151.0, std::floor(f * 2097151.0));
            code |= spread3(q) << c;
        }
        key[k] = {{cell_group ? cell_group[k] : 0, code}, (int32_t)k};
    }
    std::sort(key.begin(), key.end());
    t->perm.resize(E);
    for (int64_t k = 0; k < E; ++k) t->perm[k] = key[k].second;

    const int nblk = (int)((E + BE - 1) / BE);
    t->BE = BE;
    t->nblk = nblk;
    t->blk_e0.resize(nblk + 1);
    for (int b = 0; b <= nblk; ++b) t->blk_e0[b] = (int32_t)std::min<int64_t>((int64_t)b * BE, E);

    // pass 1, per block: its distinct dofs (ascending) with their copies, by ascending slot
    struct Blk {
        std::vector<std::pair<int32_t, int32_t>> srt;   // (dof, slot a * ne + e), sorted
        std::vector<int32_t> uq, first;                   // distinct dofs, start of each run in srt
        std::vector<int32_t> order;                       // block-local order: indices into uq
        std::vector<int32_t> ids, gid_of;                 // final ids; group of each shared dof
        int nint = 0, max_cnt = 0;
    };
    if ((int64_t)std::min<int64_t>(BE, E) * nloc > 65535) { *detail = (int64_t)BE * nloc; return BRAS_ERR_TOO_LARGE; }
    std::vector<Blk> blk(nblk);
#pragma omp parallel for schedule(dynamic, 4)
    for (int b = 0; b < nblk; ++b) {
        const int e0 = t->blk_e0[b], ne = t->blk_e0[b + 1] - e0;
        Blk& B = blk[b];
        B.srt.resize((size_t)ne * nloc);
        for (int e = 0; e < ne; ++e) {
            const int64_t K = t->perm[e0 + e];
            for (int a = 0; a < nloc; ++a) B.srt[(size_t)a * ne + e] = {l2g[K * nloc + a], a * ne + e};
        }
        std::sort(B.srt.begin(), B.srt.end());
        // (block sizes are chosen so that m = ne * nloc < 65536 and nu < 32768 hold: the
        // positions and local indices are 16-bit, bit 15 of a local index being the sign)
        for (size_t i = 0; i < B.srt.size(); ++i)
            if (i == 0 || B.srt[i].first != B.srt[i - 1].first) {
                B.uq.push_back(B.srt[i].first);
                B.first.push_back((int32_t)i);
            }
        B.first.push_back((int32_t)B.srt.size());
    }
    // pass 2: the blocks of every shared dof, ascending (CSR over dofs, filled in block order)
    std::vector<int32_t> nb_of((size_t)n + 1, 0);
    for (int b = 0; b < nblk; ++b) {
        const Blk& B = blk[b];
        for (size_t i = 0; i < B.uq.size(); ++i)
            if (B.first[i + 1] - B.first[i] != d[B.uq[i]]) nb_of[(size_t)B.uq[i] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) nb_of[i + 1] += nb_of[i];
    std::vector<int32_t> blist((size_t)nb_of[n]);
    {
        std::vector<int32_t> fill(nb_of.begin(), nb_of.end() - 1);
        for (int b = 0; b < nblk; ++b) {
            const Blk& B = blk[b];
            for (size_t i = 0; i < B.uq.size(); ++i)
                if (B.first[i + 1] - B.first[i] != d[B.uq[i]]) blist[fill[B.uq[i]]++] = b;
        }
    }
    // pass 3: groups = runs of shared dofs with equal block lists (dofs sorted by (list, id))
    std::vector<int32_t> shd;
    for (int64_t i = 0; i < n; ++i)
        if (nb_of[i + 1] > nb_of[i]) shd.push_back((int32_t)i);
    auto lst_less = [&](int32_t a, int32_t b) {
        const int32_t *pa = &blist[nb_of[a]], *ea = &blist[nb_of[a + 1]];
        const int32_t *pb = &blist[nb_of[b]], *eb = &blist[nb_of[b + 1]];
        if (std::lexicographical_compare(pa, ea, pb, eb)) return true;
        if (std::lexicographical_compare(pb, eb, pa, ea)) return false;
        return a < b;
    };
    std::sort(shd.begin(), shd.end(), lst_less);
    std::vector<int32_t> gid((size_t)n, -1);
    t->grp_size.clear();
    t->grp_cnt.clear();
    for (size_t j = 0; j < shd.size(); ++j) {
        const int32_t a = shd[j];
        const bool same = j > 0 && std::equal(&blist[nb_of[shd[j - 1]]], &blist[nb_of[shd[j - 1] + 1]],
                                              &blist[nb_of[a]], &blist[nb_of[a + 1]]);
        if (!same) {
            t->grp_size.push_back(0);
            t->grp_cnt.push_back(nb_of[a + 1] - nb_of[a]);
        }
        gid[a] = (int32_t)t->grp_size.size() - 1;
        t->grp_size.back()++;
    }
    const int64_t ngrp = (int64_t)t->grp_size.size();
    t->nsh = (int64_t)shd.size();

    // pass 4, per block: interior dofs by ascending id, then the shared ones by (group, id)
    int max_u = 0, max_ne = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(max : max_u, max_ne)
    for (int b = 0; b < nblk; ++b) {
        const int ne = t->blk_e0[b + 1] - t->blk_e0[b];
        Blk& B = blk[b];
        const int nu = (int)B.uq.size();
        for (int i = 0; i < nu; ++i)
            if (B.first[i + 1] - B.first[i] == d[B.uq[i]]) B.order.push_back(i);
        B.nint = (int)B.order.size();
        std::vector<int32_t> sh;
        for (int i = 0; i < nu; ++i)
            if (B.first[i + 1] - B.first[i] != d[B.uq[i]]) sh.push_back(i);
        std::sort(sh.begin(), sh.end(), [&](int32_t i, int32_t j) {
            const int32_t gi = gid[B.uq[i]], gj = gid[B.uq[j]];
            return gi != gj ? gi < gj : B.uq[i] < B.uq[j];
        });
        B.order.insert(B.order.end(), sh.begin(), sh.end());
        B.ids.resize(nu);
        B.gid_of.resize(nu - B.nint);
        for (int u = 0; u < nu; ++u) {
            B.ids[u] = B.uq[B.order[u]];
            if (u >= B.nint) B.gid_of[u - B.nint] = gid[B.ids[u]];
        }
        for (int i = 0; i < nu; ++i) B.max_cnt = std::max(B.max_cnt, B.first[i + 1] - B.first[i]);
        max_u = std::max(max_u, nu);
        max_ne = std::max(max_ne, ne);
    }
    t->max_u = max_u;
    t->max_ne = max_ne;
    t->max_copies = 1;
    for (int b = 0; b < nblk; ++b) t->max_copies = std::max(t->max_copies, blk[b].max_cnt);
    // packets: part A = ids | d, part B = loc, 16-byte aligned sections
    t->blk_u0.resize(nblk + 1);
    t->blk_nint.resize(nblk);
    t->blk_p0.resize(nblk);
    t->blk_pkt.resize(nblk + 1);
    t->blk_g0.assign(nblk + 1, 0);
    int64_t U = 0, P = 0, bytes = 0;
    uint32_t max_pkt = 0;
    int max_bg = 0;
    for (int b = 0; b < nblk; ++b) {
        const Blk& B = blk[b];
        const uint32_t nu = (uint32_t)B.ids.size();
        const uint32_t m = (uint32_t)(t->blk_e0[b + 1] - t->blk_e0[b]) * (uint32_t)nloc;
        uint32_t ng = 0;
        for (size_t j = 0; j < B.gid_of.size(); ++j)
            if (j == 0 || B.gid_of[j] != B.gid_of[j - 1]) ++ng;
        const uint32_t sz = pkt_size_a(nu, scatter) + pkt_size_b(m, scatter);
        t->blk_u0[b] = (int32_t)U;
        t->blk_nint[b] = B.nint;
        t->blk_p0[b] = (int32_t)P;
        t->blk_pkt[b] = bytes;
        U += nu;
        P += (int64_t)nu - B.nint;
        bytes += sz;
        max_pkt = std::max(max_pkt, sz);
        t->blk_g0[b + 1] = t->blk_g0[b] + (int32_t)ng;
        max_bg = std::max(max_bg, (int)ng);
    }
    t->blk_u0[nblk] = (int32_t)U;
    t->blk_pkt[nblk] = bytes;
    t->npart = P;
    t->U_tot = U;
    t->max_pkt = max_pkt;
    t->max_bg = max_bg;
    // the groups of each block, and the partial slots of each group in ascending block order
    t->bg_gid.resize(t->blk_g0[nblk]);
    t->bg_u.resize(t->blk_g0[nblk]);
    t->grp_slot0.assign(ngrp + 1, 0);
    for (int64_t g = 0; g < ngrp; ++g) t->grp_slot0[g + 1] = t->grp_slot0[g] + t->grp_cnt[g];
    t->grp_slots.assign(t->grp_slot0[ngrp], 0);
    {
        std::vector<int32_t> fill(t->grp_slot0.begin(), t->grp_slot0.end() - 1);
        for (int b = 0; b < nblk; ++b) {
            const Blk& B = blk[b];
            int k = t->blk_g0[b];
            for (size_t j = 0; j < B.gid_of.size(); ++j)
                if (j == 0 || B.gid_of[j] != B.gid_of[j - 1]) {
                    const int32_t g = B.gid_of[j];
                    t->bg_gid[k] = g;
                    t->bg_u[k] = B.nint + (int32_t)j;
                    t->grp_slots[fill[g]++] = t->blk_p0[b] + (int32_t)j;
                    ++k;
                }
        }
    }
    // the combine pass walks the groups: their dofs (ids, multiplicities) in group order
    t->grp_item0.assign(ngrp + 1, 0);
    for (int64_t g = 0; g < ngrp; ++g) t->grp_item0[g + 1] = t->grp_item0[g] + t->grp_size[g];
    t->sh_ids.assign(t->grp_item0[ngrp], 0);
    t->sh_d.assign(t->grp_item0[ngrp], 0);
    {
        std::vector<int32_t> fill(t->grp_item0.begin(), t->grp_item0.end() - 1);
        for (size_t j = 0; j < shd.size(); ++j) {
            const int32_t a = shd[j], g = gid[a];
            t->sh_ids[fill[g]] = a;
            t->sh_d[fill[g]++] = (uint16_t)std::min<int32_t>(d[a], 65535);
        }
    }
    t->pkt.assign((size_t)bytes, 0);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nblk; ++b) {
        const Blk& B = blk[b];
        const int ne = t->blk_e0[b + 1] - t->blk_e0[b];
        const uint32_t nu = (uint32_t)B.ids.size();
        const uint32_t m = (uint32_t)ne * (uint32_t)nloc;
        const int e0 = t->blk_e0[b];
        unsigned char* p = t->pkt.data() + t->blk_pkt[b];
        std::memcpy(p, B.ids.data(), 4 * (size_t)nu);
        uint16_t* dm = reinterpret_cast<uint16_t*>(p + pkt_off_d(nu));
        for (uint32_t u = 0; u < nu; ++u) dm[u] = (uint16_t)std::min<int32_t>(d[B.ids[u]], 65535);
        uint16_t* incoff = reinterpret_cast<uint16_t*>(p + pkt_off_incoff(nu));
        uint16_t* loc = reinterpret_cast<uint16_t*>(p + pkt_size_a(nu, scatter));
        uint16_t* pos = loc + pkt_off_pos(m) / 2;
        // dof-sorted order (scatter tables): the dofs in block-local order u, each dof's copies
        // by ascending slot
        uint32_t off = 0;
        for (uint32_t u = 0; u < nu; ++u) {
            const int i = B.order[u];
            if (scatter) incoff[u] = (uint16_t)off;
            for (int s = B.first[i]; s < B.first[i + 1]; ++s) {
                const int slot = B.srt[s].second, a = slot / ne, e = slot % ne;
                const int64_t K = t->perm[e0 + e];
                const bool neg = signs && signs[K * nloc + a] < 0;
                loc[slot] = (uint16_t)(u | (neg ? 0x8000u : 0u));
                if (scatter) pos[slot] = (uint16_t)off;
                ++off;
            }
        }
        if (scatter) incoff[nu] = (uint16_t)off;
    }
    return BRAS_OK;
}

}  // namespace bras
