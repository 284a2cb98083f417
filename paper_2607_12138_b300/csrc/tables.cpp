// Host construction of the deterministic scatter tables (setup time, not timed).
//
// The BRAS apply D^{-1} P^T M_br^{-1} P D^{-1} (Eq. mhatinvbras_def) and the mass apply
// P^T M_br P (Eq. M_PMbrP) both end in the transpose of the signed gather P: every conforming
// dof sums the contributions of its broken copies.  These tables let one thread block do
// that sum in on-chip memory for the dofs whose copies all live in its cells, and hand the
// few dofs on block boundaries to a second, fixed-order pass -- no floating-point atomics.
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
                 int64_t* detail, const int32_t* cell_group) {
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

    struct Blk {
        std::vector<int32_t> ids;
        std::vector<uint16_t> incoff, inc, loc;
        int nint = 0;
    };
    std::vector<Blk> blk(nblk);
    int max_u = 0, max_ne = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(max : max_u, max_ne)
    for (int b = 0; b < nblk; ++b) {
        const int e0 = t->blk_e0[b], ne = t->blk_e0[b + 1] - e0;
        std::vector<std::pair<int32_t, int32_t>> pr((size_t)ne * nloc);   // (dof, slot)
        for (int e = 0; e < ne; ++e) {
            const int64_t K = t->perm[e0 + e];
            for (int a = 0; a < nloc; ++a) pr[(size_t)a * ne + e] = {l2g[K * nloc + a], a * ne + e};
        }
        std::vector<std::pair<int32_t, int32_t>> srt(pr);
        std::sort(srt.begin(), srt.end());
        // unique dofs with in-block copy counts
        std::vector<int32_t> uq, first;
        for (size_t i = 0; i < srt.size(); ++i)
            if (i == 0 || srt[i].first != srt[i - 1].first) { uq.push_back(srt[i].first); first.push_back((int32_t)i); }
        first.push_back((int32_t)srt.size());
        const int nu = (int)uq.size();
        // interior first, then shared, each in ascending dof id (neighbouring threads touch
        // neighbouring entries of x and y)
        std::vector<int32_t> order;
        order.reserve(nu);
        for (int i = 0; i < nu; ++i) if (first[i + 1] - first[i] == d[uq[i]]) order.push_back(i);
        const int nint = (int)order.size();
        for (int i = 0; i < nu; ++i) if (first[i + 1] - first[i] != d[uq[i]]) order.push_back(i);
        std::vector<int32_t> uidx(nu);
        Blk& B = blk[b];
        B.nint = nint;
        B.ids.resize(nu);
        B.incoff.resize(nu + 1);
        B.inc.resize((size_t)ne * nloc);
        int off = 0;
        for (int u = 0; u < nu; ++u) {
            const int i = order[u];
            uidx[i] = u;
            B.ids[u] = uq[i];
            B.incoff[u] = (uint16_t)off;
            for (int s = first[i]; s < first[i + 1]; ++s) B.inc[off++] = (uint16_t)srt[s].second;
        }
        B.incoff[nu] = (uint16_t)off;
        // loc: block-local index of each broken copy, sign in bit 15
        B.loc.resize((size_t)ne * nloc);
        for (int i = 0; i < nu; ++i)
            for (int s = first[i]; s < first[i + 1]; ++s) {
                const int slot = srt[s].second, a = slot / ne, e = slot % ne;
                const int64_t K = t->perm[e0 + e];
                const bool neg = signs && signs[K * nloc + a] < 0;
                B.loc[slot] = (uint16_t)(uidx[i] | (neg ? 0x8000 : 0));
            }
        max_u = std::max(max_u, nu);
        max_ne = std::max(max_ne, ne);
    }
    t->max_u = max_u;
    t->max_ne = max_ne;
    // packets: part A = ids | d | incoff, part B = loc | inc, 16-byte aligned sections
    t->blk_u0.resize(nblk + 1);
    t->blk_nint.resize(nblk);
    t->blk_p0.resize(nblk);
    t->blk_pkt.resize(nblk + 1);
    int64_t U = 0, P = 0, bytes = 0;
    uint32_t max_pkt = 0;
    for (int b = 0; b < nblk; ++b) {
        const uint32_t nu = (uint32_t)blk[b].ids.size();
        const uint32_t m = (uint32_t)(t->blk_e0[b + 1] - t->blk_e0[b]) * (uint32_t)nloc;
        const uint32_t sz = pkt_size_a(nu) + pkt_size_b(m);
        t->blk_u0[b] = (int32_t)U;
        t->blk_nint[b] = blk[b].nint;
        t->blk_p0[b] = (int32_t)P;
        t->blk_pkt[b] = bytes;
        U += nu;
        P += (int64_t)nu - blk[b].nint;
        bytes += sz;
        max_pkt = std::max(max_pkt, sz);
    }
    t->blk_u0[nblk] = (int32_t)U;
    t->blk_pkt[nblk] = bytes;
    t->npart = P;
    t->U_tot = U;
    t->max_pkt = max_pkt;
    t->pkt.assign((size_t)bytes, 0);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nblk; ++b) {
        const Blk& B = blk[b];
        const uint32_t nu = (uint32_t)B.ids.size();
        const uint32_t m = (uint32_t)B.loc.size();
        unsigned char* p = t->pkt.data() + t->blk_pkt[b];
        std::memcpy(p, B.ids.data(), 4 * (size_t)nu);
        uint16_t* dm = reinterpret_cast<uint16_t*>(p + pkt_off_d(nu));
        for (uint32_t u = 0; u < nu; ++u) dm[u] = (uint16_t)std::min<int32_t>(d[B.ids[u]], 65535);
        std::memcpy(p + pkt_off_incoff(nu), B.incoff.data(), 2 * (size_t)(nu + 1));
        const uint32_t sa = pkt_size_a(nu);
        std::memcpy(p + sa, B.loc.data(), 2 * (size_t)m);
        // position of every broken copy in the dof-sorted order (the inverse of the incidence
        // list): a cell writes its result for copy (a, e) there, and each dof then sums one
        // contiguous run
        uint16_t* pos = reinterpret_cast<uint16_t*>(p + sa + pad16(2u * m));
        for (uint32_t s = 0; s < m; ++s) pos[B.inc[s]] = (uint16_t)s;
    }
    // shared dofs: partial slots in ascending block order per dof
    std::vector<std::pair<int32_t, int32_t>> sh;   // (dof, slot)
    sh.reserve(P);
    for (int b = 0; b < nblk; ++b) {
        const Blk& B = blk[b];
        for (size_t u = B.nint; u < B.ids.size(); ++u)
            sh.push_back({B.ids[u], t->blk_p0[b] + (int32_t)(u - B.nint)});
    }
    std::stable_sort(sh.begin(), sh.end(), [](auto& x, auto& y) { return x.first < y.first; });
    t->sh_ids.clear();
    t->sh_off.clear();
    t->sh_slots.resize(sh.size());
    for (size_t i = 0; i < sh.size(); ++i) {
        if (i == 0 || sh[i].first != sh[i - 1].first) {
            t->sh_ids.push_back(sh[i].first);
            t->sh_off.push_back((int32_t)i);
        }
        t->sh_slots[i] = sh[i].second;
    }
    t->sh_off.push_back((int32_t)sh.size());
    return BRAS_OK;
}

}  // namespace bras
