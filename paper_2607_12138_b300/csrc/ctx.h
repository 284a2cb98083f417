// Internal context of libbras (not part of the ABI).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bras.h"

namespace bras {

struct PcgWork;

// ---- scatter tables ---------------------------------------------------------------
// Cells are reordered along a Morton curve of their centroids and cut into blocks of at
// most BE consecutive cells.  Block b owns cells [blk_e0[b], blk_e0[b+1]) and nu_b =
// blk_u0[b+1] - blk_u0[b] block-local dofs: first the dofs all of whose broken copies lie
// inside the block ("interior", blk_nint[b] of them, ascending global id), then the others
// ("shared"), grouped.  Its table packet (byte offset blk_pkt[b], layout in packet.h) holds
// the dof ids, multiplicities and local indices with signs.
// A group is the set of shared dofs whose copies lie in one and the same set of blocks
// (grp_cnt[g] blocks, grp_size[g] dofs); every member block lists the group's dofs
// contiguously, by ascending global id.  Shared dof u of block b leaves its partial sum in
// slot blk_p0[b] + u - nint_b; grp_slots[grp_slot0[g] + k] is the slot of the group's first
// dof in its k-th block (ascending block order), so the partials of the group's dof i sit at
// grp_slots[...] + i.  Block b's groups are bg_gid[blk_g0[b] .. blk_g0[b+1]) with their first
// block-local dof bg_u[...].  The combine pass walks the groups (grp_item0, sh_ids, sh_d:
// the group's dofs in order, with their multiplicities) and sums each dof's partials in the
// fixed block order.
struct HostTables {
    int BE = 256, nblk = 0, max_u = 0, max_ne = 0;
    uint32_t max_pkt = 0;
    std::vector<int32_t> perm, blk_e0, blk_u0, blk_nint, blk_p0;
    std::vector<int32_t> grp_size, grp_cnt, grp_slot0, grp_slots, blk_g0, bg_gid, bg_u;
    std::vector<int32_t> grp_item0, sh_ids;   // combine pass: group g's dofs are sh_ids[grp_item0[g] ..]
    std::vector<uint16_t> sh_d;               // and their multiplicities
    std::vector<int64_t> blk_pkt;
    std::vector<unsigned char> pkt;
    std::vector<double> dinv;
    int64_t npart = 0, U_tot = 0, nsh = 0;
    int max_bg = 0;       // most groups of one block
    int max_copies = 1;   // most copies of one dof inside one block
};

// scatter = true: the packets also carry the dof-sorted positions and run offsets (blocks of
// streamed cell matrices); false: local indices only (H1, fixed-point sums)
int build_tables(const int32_t* l2g, const int8_t* signs, int64_t E, int nloc, int64_t n,
                 const double* coords, const int32_t* cells, int dim, int BE, HostTables* t,
                 int64_t* detail, const int32_t* cell_group = nullptr, bool scatter = false);

}  // namespace bras

struct bras_ctx {
    int dim = 0, space = 0, order = 0, nloc = 0, ncomp = 0;
    int64_t E = 0, n = 0, nvert = 0;
    int BE = 256, nblk = 0, max_u = 0, max_ne = 0;
    int precisions = 0, max_nrhs = 1;
    // fixed-point dof sums: product bound placed at 2^fx_top; exponent bounds of the local
    // operators' row abs-sums (mass, BRAS)
    int fx_top = 43, fx_lo = 22, fx_top_df = 50, fx_lo_df = 24, fx_top64 = 56, er_mass = 0, er_bras = 0;
    int64_t U_tot = 0, npart = 0, nsh = 0;
    int64_t Epad = 0;   // padded cell count of the packed (SoA) per-cell matrices
    int npk = 0;        // nloc (nloc + 1) / 2
    int bf16_fixed = 0; // cells whose bf16-rounded inverse needed a diagonal shift
    int tune_count = 0; // block sizes the autotuner timed, and their BRAS apply times
    int tune_be[8] = {0};
    float tune_us[8] = {0};

    // scatter tables (device)
    int32_t *blk_e0 = nullptr, *blk_u0 = nullptr, *blk_nint = nullptr, *blk_p0 = nullptr;
    // shared dofs by group, for the combine pass
    int2* sh_items = nullptr;    // (global dof, group)
    uint16_t* sh_d = nullptr;    // multiplicity
    int4* grp_rec = nullptr;     // (first item, block count, first slot entry, 0)
    int32_t* grp_slots = nullptr;
    int64_t ngrp = 0;
    int32_t *perm = nullptr;
    int64_t* blk_pkt = nullptr;
    unsigned char* pkt = nullptr;
    uint32_t max_pkt = 0;

    // many right-hand sides on streamed cell matrices (max_nrhs >= 16, n_loc <= 48): maps in
    // internal cell order (bit 31 = sign of P), dof-sorted copy slots, first slot of each dof
    int32_t* mr_l2g = nullptr;
    int32_t* mr_slot = nullptr;
    int64_t* mr_off = nullptr;

    // per dof
    double* dinv64 = nullptr;
    float* dinv32 = nullptr;
    double* diag64 = nullptr;
    float* diag32 = nullptr;

    // geometry (internal cell order)
    double* absdet = nullptr;    // |det J_K|
    double* rho = nullptr;       // weights
    double* metric = nullptr;    // [6][E] symmetric Piola metric (vector spaces)

    // H1: reference mass and inverse, per-cell factors
    double *Mref64 = nullptr, *Minvref64 = nullptr;
    float *Mref32 = nullptr, *Minvref32 = nullptr;
    double *mscale64 = nullptr, *bscale64 = nullptr;
    float *mscale32 = nullptr, *bscale32 = nullptr;

    // H(curl)/H(div): packed lower-triangular-by-rows symmetric matrices, SoA [npk][Epad]
    double* Rref = nullptr;      // [ncomp*ncomp][nloc][nloc] reference blocks
    double *Mpk64 = nullptr, *Minvpk64 = nullptr;
    float *Mpk32 = nullptr, *Minvpk32 = nullptr;
    __nv_bfloat16* Minvpkbf = nullptr;
    float2* Mpkdf = nullptr;     // Mpk64 as (hi, lo) float pairs (many-right-hand-side contexts)

    // H1 tensor-core path: reference matrices pre-split (TF32 big | remainder) and laid out
    // as the GEMM's shared-memory B operand
    bool use_tc = false;
    unsigned char *btile_mass = nullptr, *btile_bras = nullptr;

    // mixed Poisson Schur complement (RT_k / DG_{k-1} on tetrahedra), caller's cell order
    int nq = 0;                  // DG_{k-1} dofs per cell
    double* Bdiv64 = nullptr;    // [nq][nloc] reference divergence block
    float* Bdiv32 = nullptr;
    int32_t* l2g_user = nullptr; // [E][nloc]
    int8_t* sgn_user = nullptr;  // [E][nloc] sign of P times sign(det J_K)
    int32_t* cpos = nullptr;     // [E][nloc] slot of each copy in dof-sorted order (cell, local index ascending)
    int64_t* coff = nullptr;     // [n + 1] first slot of each dof
    void* schur_ws = nullptr;    // copies [E * nloc], then two dof vectors (8-byte entries)
    size_t schur_ws_bytes = 0;

    // workspace
    void* part = nullptr;        // partial sums of shared dofs [npart * nrhs] (double)
    size_t part_bytes = 0;
    int* status = nullptr;       // device status words
    bras::PcgWork* pcg = nullptr;

    // batched multi-mesh contexts: mesh m owns dofs [dof_off[m], dof_off[m+1]); the vector
    // kernels of the solve work on segments of one mesh each (seg_beg[s]..seg_beg[s+1]),
    // mesh m owning segments [mseg[m], mseg[m+1])
    int n_mesh = 1;
    int nseg = 0;
    std::vector<int64_t> dof_off;
    int32_t* seg_mesh = nullptr;
    int64_t* seg_beg = nullptr;
    int32_t* mseg = nullptr;

    std::vector<void*> owned;    // every device allocation, freed by bras_destroy
};
