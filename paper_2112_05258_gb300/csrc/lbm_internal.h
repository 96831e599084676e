// Internal data layout shared by the host layout builder, the kernels and the
// C-ABI entry points of liblbm.  Nothing here is part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

struct lbm_config_s;

namespace lbm {

constexpr int NQ = 19;
constexpr int MAX_BC = 8;
constexpr int CHUNK = 32;  // cells per chunk of the chunk-to-row table
constexpr int BC_CHUNK = 256;  // first-layer cells or links per CTA of the boundary kernels

// D3Q19 velocity set in the public order (rest, +-x, +-y, +-z, 12 edges).
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
// index of the neighbour row (y - ey, z - ez) a population i is pulled from
__host__ __device__ constexpr int nbk(int i) { return (1 - cy(i)) + 3 * (1 - cz(i)); }

// Offset of population i of stored cell c in a population buffer of N cells:
// structure of arrays, f[i][c] (the stream-collide kernel addresses the same
// layout through one base pointer per direction).  19 N < 2^31 keeps
// offsets in 32 bits.
__host__ __device__ inline uint32_t pidx(int i, uint32_t c, uint32_t N) { return (uint32_t)i * N + c; }
inline int64_t population_cells(int64_t N) { return N; }

// Per-cell flag word: bits 0..18 = the pull source of direction i is a rigid
// wall (halfway bounce-back: read the opposite population of the own cell).
enum : uint32_t {
    FL_ACTIVE = 1u << 24,  // fluid cell updated by stream-collide
    FL_BAND = 1u << 25,    // carries an immersed-boundary force density b
    FL_XF = 1u << 26,      // first fluid layer of a 0D boundary: macros go to aux
    FL_BNODE = 1u << 27,   // storage slot of a 0D boundary node (ghost populations)
    FL_BBMASK = (1u << 19) - 1u
};

// One row of stored cells: the cells x0 .. x0+len-1 at fixed (y, z) of one
// instance.  nb[k] = off(r') - x0(r') of the neighbour row r' at
// (y + sy, z + sz) with k = (1 + sy) + 3 (1 + sz), or 0 when absent, so the
// compact index of the stored cell (x', y + sy, z + sz) is nb[k] + x'.
// 64 bytes, so that a kernel reads a whole row entry with four 16-byte loads.
struct alignas(16) RowInfo {
    int32_t off;
    int32_t x0;
    int32_t len;
    int32_t inst;
    int32_t y, z;
    int32_t nb[9];
    int32_t pad;
};
static_assert(sizeof(RowInfo) == 64, "row entry is four 16-byte words");

struct InstParam {
    double tau;
    double omega;   // 1/tau
    int nx, ny, nz;
    int rowid_off;  // offset of this instance's (ny*nz) row-id table
    int q_scale;
    int ib_off, n_ib;
    int bc_first, n_bc;
    double alpha, beta, ms;
    double inv_ms;  // 1/ms (FP64 division is slow on the device)
    float alpha_f, beta_f, inv_ms_f;  // the same rounded to FP32 (wall-node state in FP32)
};

enum { BC_VELOCITY = 0, BC_RCR = 1, BC_LV = 2, BC_PRESSURE = 3 };

struct BcParam {
    int kind, axis, sign, inst;
    int n_xf, xf_off;
    int n_links, link_off;
    int n_nodes, node_off;  // profile rows (velocity kind)
    int period, etab_off;   // elastance table (LV kind)
    int q_scale;
    int local;              // index of this boundary within its instance
    int red_off, n_red;     // partial sums of the first-layer reduction
    double par[8];
};

struct BcState {
    double Q, Qu, Pbar;     // at t_n
    double Pw, Pv;          // chamber / ventricle gauge pressure
    double valve_open, Td;
    double Pstar_gauge;
};

// Host-side layout produced from the node arrays.
struct Layout {
    int64_t n_stored = 0, n_fluid = 0, n_box = 0;
    std::vector<RowInfo> rows;          // + one sentinel row with off = n_stored
    std::vector<int32_t> chunk_row;     // per CHUNK of 32 cells: {row of its first cell, mask of the
                                        // lanes 1..31 whose cell begins a new row}, interleaved
    std::vector<uint32_t> flags;        // per stored cell
    std::vector<int64_t> cell_box;      // per stored cell: box index within its instance
    std::vector<int32_t> cell_inst;     // per stored cell
    std::vector<int32_t> rowid;         // per instance (ny*nz), concatenated
    std::vector<InstParam> inst;
    std::vector<int64_t> inst_cell_begin, inst_cell_end;
    std::vector<int64_t> inst_fluid;
    // boundaries
    std::vector<BcParam> bc;
    std::vector<int32_t> xf;            // compact cells of first fluid layers
    std::vector<int32_t> lk_xb, lk_xf;  // link slots
    std::vector<uint8_t> lk_i;
    std::vector<int32_t> lk_node, lk_xfi;
    std::vector<double> profile;        // 3 per node (velocity kinds)
    std::vector<double> etab;           // 2 per entry (LV kinds)
    std::vector<int32_t> red_bc, red_chunk, app_bc, app_chunk;  // boundary kernel block tables
    int64_t n_partial = 0;
    // immersed boundary
    std::vector<int32_t> band;          // compact cells flagged FL_BAND
    // per wall node, around its reference cell i0 = floor(X0 - 0.5): compact
    // index of x = 0 on the 36 lattice lines y = i0y - 2 .. +3, z = i0z - 2 .. +3
    // (line jy + 6 jz), and a 216-bit mask of the fluid cells of that 6^3 box
    // (bit jx + 6 (jy + 6 jz), x = i0x - 2 + jx), as 4 x 64-bit words
    std::vector<int32_t> ib_lines;
    std::vector<uint64_t> ib_mask;
    std::vector<int32_t> ib_ref;        // i0 per node (3 ints)
    std::vector<float> ib_g0;           // X0 - 1/2 - i0 per node (3, in [0, 1)), rounded to FP32
    std::vector<double> ib_X0, ib_dA, ib_ks;
    std::vector<uint8_t> ib_pinned;     // 0 spring, 1 pinned, 2 moved by its filament
    // filaments: global wall-node lists, first entry and count per filament, (ds, Eh, EI)
    std::vector<int32_t> fil_nodes, fil_start, fil_count;
    std::vector<double> fil_par;
    int max_fil = 0;
    // slabs of the wall-node pipeline (empty: one launch per kernel per step):
    // slab s holds the stored cells [slab_cell[s], slab_cell[s+1]), the band
    // entries [slab_band[s], slab_band[s+1]) and the wall nodes
    // node_order[slab_node[s] .. slab_node[s+1])
    std::vector<int32_t> slab_cell, slab_band, slab_node, node_order;
};

// Cuts the compact cell range into about `want` slabs for the pipelined step
// (see build_slabs in lbm_layout.cu); leaves the slab tables empty when the
// lattice has no wall nodes, has filaments, or gives fewer than 3 slabs.
void build_slabs(Layout &L, int want);

}  // namespace lbm
