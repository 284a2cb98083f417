// Test harness (host only): runs the library's block-table builder (csrc/tables.cpp) on a mesh
// read from a binary file and writes every table it produced, for the CPU tests to check.
//
// Input (little endian): int64 E, int32 nloc, int64 n, int32 dim, int32 BE, int64 nvert,
//   int32 has_signs, int32 has_groups, int32 scatter, int32 l2g[E*nloc], [int8 signs[E*nloc]],
//   double coords[nvert*dim], int32 cells[E*(dim+1)], [int32 groups[E]].
// Output: int32 rc, int64 detail, and for rc == 0: int32 BE, nblk, max_u, max_ne, max_bg, max_copies,
//   uint32 max_pkt, int64 npart, U_tot, nsh, then the arrays perm, blk_e0, blk_u0, blk_nint,
//   blk_p0, grp_size, grp_cnt, grp_slot0, grp_slots, blk_g0, bg_gid, bg_u, grp_item0, sh_ids
//   (int32), sh_d (uint16), blk_pkt (int64), pkt (uint8), dinv (double), each preceded by its
//   int64 length.
#include <cstdio>
#include <vector>

#include "ctx.h"

namespace {

template <typename T> bool rd(FILE* f, T* p, size_t n) { return fread(p, sizeof(T), n, f) == n; }
template <typename T> void wr(FILE* f, const T& v) { fwrite(&v, sizeof(T), 1, f); }
template <typename T> void wr_vec(FILE* f, const std::vector<T>& v) {
    const int64_t n = (int64_t)v.size();
    wr(f, n);
    if (n) fwrite(v.data(), sizeof(T), v.size(), f);
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 2;
    int64_t E = 0, n = 0, nvert = 0;
    int32_t nloc = 0, dim = 0, BE = 0, has_signs = 0, has_groups = 0, scatter = 0;
    bool ok = rd(in, &E, 1) && rd(in, &nloc, 1) && rd(in, &n, 1) && rd(in, &dim, 1) && rd(in, &BE, 1) &&
              rd(in, &nvert, 1) && rd(in, &has_signs, 1) && rd(in, &has_groups, 1) && rd(in, &scatter, 1);
    std::vector<int32_t> l2g(ok ? E * nloc : 0), cells(ok ? E * (dim + 1) : 0), groups;
    std::vector<int8_t> signs;
    std::vector<double> coords(ok ? nvert * dim : 0);
    ok = ok && rd(in, l2g.data(), l2g.size());
    if (ok && has_signs) {
        signs.resize(l2g.size());
        ok = rd(in, signs.data(), signs.size());
    }
    ok = ok && rd(in, coords.data(), coords.size()) && rd(in, cells.data(), cells.size());
    if (ok && has_groups) {
        groups.resize(E);
        ok = rd(in, groups.data(), groups.size());
    }
    fclose(in);
    if (!ok) return 2;

    bras::HostTables t;
    int64_t detail = -1;
    const int rc = bras::build_tables(l2g.data(), has_signs ? signs.data() : nullptr, E, nloc, n, coords.data(),
                                      cells.data(), dim, BE, &t, &detail, has_groups ? groups.data() : nullptr,
                                      scatter != 0);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 2;
    wr(out, (int32_t)rc);
    wr(out, detail);
    if (rc == 0) {
        wr(out, (int32_t)t.BE);
        wr(out, (int32_t)t.nblk);
        wr(out, (int32_t)t.max_u);
        wr(out, (int32_t)t.max_ne);
        wr(out, (int32_t)t.max_bg);
        wr(out, (int32_t)t.max_copies);
        wr(out, (uint32_t)t.max_pkt);
        wr(out, (int64_t)t.npart);
        wr(out, (int64_t)t.U_tot);
        wr(out, (int64_t)t.nsh);
        for (const auto* v : {&t.perm, &t.blk_e0, &t.blk_u0, &t.blk_nint, &t.blk_p0, &t.grp_size, &t.grp_cnt,
                              &t.grp_slot0, &t.grp_slots, &t.blk_g0, &t.bg_gid, &t.bg_u, &t.grp_item0, &t.sh_ids})
            wr_vec(out, *v);
        wr_vec(out, t.sh_d);
        wr_vec(out, t.blk_pkt);
        wr_vec(out, t.pkt);
        wr_vec(out, t.dinv);
    }
    fclose(out);
    return 0;
}
