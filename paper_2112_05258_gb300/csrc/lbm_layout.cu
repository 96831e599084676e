// Host-side construction of the compact row layout from node-type arrays.
//
// Every instance is cut into rows of constant (y, z); a row stores the cells
// from its first to its last non-wall node (fluid or 0D boundary node), so
// solid cells outside the vessel cost neither memory nor bandwidth.  Rows of
// all instances are concatenated into one compact cell index space, which is
// how a batch of instances is packed into one launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <unordered_map>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {

static std::string fmt(const char *f, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

std::string build_layout(const lbm_config *cfg, Layout &L) {
    const int ni = cfg->n_instances;
    int64_t cell = 0;
    L.inst.resize(ni);
    L.inst_cell_begin.resize(ni);
    L.inst_cell_end.resize(ni);
    L.inst_fluid.resize(ni);
    for (int q = 0; q < ni; q++) {
        const lbm_instance_desc &d = cfg->inst[q];
        const int nx = d.nx, ny = d.ny, nz = d.nz;
        const int64_t nbox = (int64_t)nx * ny * nz;
        const uint8_t *node = d.node;
        InstParam &ip = L.inst[q];
        ip.tau = d.tau;
        ip.omega = 1.0 / d.tau;
        ip.nx = nx;
        ip.ny = ny;
        ip.nz = nz;
        ip.rowid_off = (int)L.rowid.size();
        ip.q_scale = d.q_scale;
        ip.n_bc = d.n_bc;
        ip.alpha = d.ib_alpha;
        ip.beta = d.ib_beta;
        ip.ms = d.ib_ms;
        ip.inv_ms = d.ib_ms > 0 ? 1.0 / d.ib_ms : 0.0;
        ip.alpha_f = (float)ip.alpha;
        ip.beta_f = (float)ip.beta;
        ip.inv_ms_f = (float)ip.inv_ms;
        L.n_box += nbox;
        L.inst_cell_begin[q] = cell;
        const int row_base = (int)L.rows.size();
        L.rowid.resize(L.rowid.size() + (size_t)ny * nz, -1);
        int32_t *rowid = &L.rowid[ip.rowid_off];
        // rows
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++) {
                const uint8_t *r = node + (int64_t)nx * (y + (int64_t)ny * z);
                int first = -1, last = -1;
                for (int x = 0; x < nx; x++)
                    if (r[x] != 1) {
                        if (first < 0) first = x;
                        last = x;
                    }
                if (first < 0) continue;
                RowInfo ri;
                memset(&ri, 0, sizeof ri);
                ri.off = (int32_t)cell;
                ri.x0 = first;
                ri.len = last - first + 1;
                ri.inst = q;
                ri.y = y;
                ri.z = z;
                rowid[y + ny * z] = (int32_t)L.rows.size();
                L.rows.push_back(ri);
                cell += ri.len;
                if (cell > INT32_MAX - 64) return "lattice too large for 32-bit cell indices";
            }
        // neighbour-row bases
        for (size_t r = row_base; r < L.rows.size(); r++) {
            RowInfo &ri = L.rows[r];
            for (int sz = -1; sz <= 1; sz++)
                for (int sy = -1; sy <= 1; sy++) {
                    int yy = ri.y + sy, zz = ri.z + sz;
                    int k = (1 + sy) + 3 * (1 + sz);
                    ri.nb[k] = 0;
                    if (yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                    int rr = rowid[yy + ny * zz];
                    if (rr >= 0) ri.nb[k] = L.rows[rr].off - L.rows[rr].x0;
                }
        }
        L.inst_cell_end[q] = cell;
    }
    L.n_stored = cell;
    // sentinel row
    RowInfo sent;
    memset(&sent, 0, sizeof sent);
    sent.off = (int32_t)cell;
    sent.inst = -1;
    L.rows.push_back(sent);
    // chunk -> {row of the first cell, lanes starting a new row}
    const int64_t nchunk = (cell + CHUNK - 1) / CHUNK;
    L.chunk_row.assign(2 * nchunk, 0);
    {
        size_t r = 0;
        for (int64_t c = 0; c < nchunk; c++) {
            const int64_t first = c * CHUNK;
            while (L.rows[r + 1].off <= first) r++;
            L.chunk_row[2 * c] = (int32_t)r;
            uint32_t mask = 0;
            for (size_t rr = r + 1; rr + 1 < L.rows.size() && L.rows[rr].off < first + CHUNK; rr++)
                mask |= 1u << (L.rows[rr].off - first);
            L.chunk_row[2 * c + 1] = (int32_t)mask;
        }
    }
    // per-cell flags, box index, instance
    L.flags.assign(cell, 0u);
    L.cell_box.assign(cell, 0);
    L.cell_inst.assign(cell, 0);
    for (size_t r = 0; r + 1 < L.rows.size(); r++) {
        const RowInfo &ri = L.rows[r];
        const lbm_instance_desc &d = cfg->inst[ri.inst];
        const int nx = d.nx, ny = d.ny, nz = d.nz;
        for (int k = 0; k < ri.len; k++) {
            const int x = ri.x0 + k, y = ri.y, z = ri.z;
            const int64_t c = ri.off + k;
            const int64_t b = x + (int64_t)nx * (y + (int64_t)ny * z);
            L.cell_box[c] = b;
            L.cell_inst[c] = ri.inst;
            const uint8_t code = d.node[b];
            uint32_t fl = 0;
            if (code == 0) {
                fl |= FL_ACTIVE;
                for (int i = 1; i < NQ; i++) {
                    int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
                    bool wall = sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz ||
                                d.node[sx + (int64_t)nx * (sy + (int64_t)ny * sz)] == 1;
                    if (wall) fl |= (1u << i);
                }
            } else if (code >= 2) {
                fl |= FL_BNODE;
            }
            L.flags[c] = fl;
        }
    }
    // verify every pull source against the box (guards the kernels' indexing)
    for (int q = 0; q < ni; q++) {
        const lbm_instance_desc &d = cfg->inst[q];
        const InstParam &ip = L.inst[q];
        std::vector<int32_t> box2c((size_t)d.nx * d.ny * d.nz, -1);
        for (int64_t c = L.inst_cell_begin[q]; c < L.inst_cell_end[q]; c++) box2c[L.cell_box[c]] = (int32_t)c;
        int64_t nfl = 0;
        for (int64_t c = L.inst_cell_begin[q]; c < L.inst_cell_end[q]; c++) {
            uint32_t fl = L.flags[c];
            if (!(fl & FL_ACTIVE)) continue;
            nfl++;
            int64_t b = L.cell_box[c];
            int x = (int)(b % d.nx), y = (int)((b / d.nx) % d.ny), z = (int)(b / ((int64_t)d.nx * d.ny));
            int r = L.rowid[ip.rowid_off + y + d.ny * z];
            const RowInfo &ri = L.rows[r];
            if (ri.off + (x - ri.x0) != c) return "layout self-check failed (own index)";
            for (int i = 1; i < NQ; i++) {
                if (fl & (1u << i)) continue;
                int sx = x - cx(i), sy = y - cy(i), sz = z - cz(i);
                int64_t src = (int64_t)ri.nb[nbk(i)] + sx;
                int64_t want = box2c[sx + (int64_t)d.nx * (sy + (int64_t)d.ny * sz)];
                if (want < 0 || src != want) return fmt("layout self-check failed at cell %lld dir %lld", c, i);
            }
        }
        L.inst_fluid[q] = nfl;
        L.n_fluid += nfl;
    }
    // boundaries: nodes in raster order, links (x_b, i) with x_b + e_i fluid,
    // first fluid layer = link targets in order of first appearance
    for (int q = 0; q < ni; q++) {
        const lbm_instance_desc &d = cfg->inst[q];
        const int nx = d.nx, ny = d.ny, nz = d.nz;
        const int64_t nbox = (int64_t)nx * ny * nz;
        std::vector<int32_t> box2c((size_t)nbox, -1);
        for (int64_t c = L.inst_cell_begin[q]; c < L.inst_cell_end[q]; c++) box2c[L.cell_box[c]] = (int32_t)c;
        if (d.n_bc < 0 || d.n_bc > MAX_BC) return "n_bc out of range";
        L.inst[q].bc_first = (int)L.bc.size();
        for (int k = 0; k < d.n_bc; k++) {
            const lbm_boundary_desc &bd = d.bc[k];
            BcParam bp;
            memset(&bp, 0, sizeof bp);
            bp.kind = bd.kind;
            bp.axis = bd.axis;
            bp.sign = bd.sign;
            bp.inst = q;
            bp.local = k;
            bp.q_scale = d.q_scale;
            for (int p = 0; p < bd.n_params && p < 8; p++) bp.par[p] = bd.params[p];
            bp.xf_off = (int)L.xf.size();
            bp.link_off = (int)L.lk_xb.size();
            bp.node_off = (int)(L.profile.size() / 3);
            const uint8_t code = (uint8_t)(2 + k);
            std::unordered_map<int64_t, int32_t> xf_of;  // box index -> first-layer index
            int node_count = 0;
            std::vector<int64_t> xf_box;
            for (int64_t b = 0; b < nbox; b++) {
                if (d.node[b] != code) continue;
                int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / ((int64_t)nx * ny));
                for (int i = 1; i < NQ; i++) {
                    int tx = x + cx(i), ty = y + cy(i), tz = z + cz(i);
                    if (tx < 0 || tx >= nx || ty < 0 || ty >= ny || tz < 0 || tz >= nz) continue;
                    int64_t t = tx + (int64_t)nx * (ty + (int64_t)ny * tz);
                    if (d.node[t] != 0) continue;
                    int32_t xfi;
                    auto it = xf_of.find(t);
                    if (it != xf_of.end()) {
                        xfi = it->second;
                    } else {
                        xfi = (int32_t)xf_box.size();
                        xf_of.emplace(t, xfi);
                        xf_box.push_back(t);
                        L.xf.push_back(box2c[t]);
                        L.flags[box2c[t]] |= FL_XF;
                    }
                    L.lk_xb.push_back(box2c[b]);
                    L.lk_xf.push_back(box2c[t]);
                    L.lk_i.push_back((uint8_t)i);
                    L.lk_node.push_back(node_count);
                    L.lk_xfi.push_back(xfi);
                }
                node_count++;
            }
            bp.n_nodes = node_count;
            bp.n_xf = (int)xf_box.size();
            bp.n_links = (int)L.lk_xb.size() - bp.link_off;
            if (bp.n_xf == 0) return fmt("boundary %lld of instance %lld has no fluid neighbour", k, q);
            if (bd.kind == BC_VELOCITY) {
                if (bd.n_profile != node_count || !bd.profile) return "velocity profile length differs from node count";
                L.profile.insert(L.profile.end(), bd.profile, bd.profile + 3 * node_count);
            }
            if (bd.kind == BC_LV) {
                if (bd.period <= 0 || !bd.elastance) return "LV boundary needs an elastance table";
                bp.period = bd.period;
                bp.etab_off = (int)(L.etab.size() / 2);
                L.etab.insert(L.etab.end(), bd.elastance, bd.elastance + 2 * (size_t)bd.period);
            }
            L.bc.push_back(bp);
        }
    }
    // block tables of the boundary kernels
    for (size_t b = 0; b < L.bc.size(); b++) {
        BcParam &bp = L.bc[b];
        bp.n_red = std::max(1, (bp.n_xf + BC_CHUNK - 1) / BC_CHUNK);  // one at least: it takes the 0D step
        bp.red_off = (int)L.n_partial;
        L.n_partial += bp.n_red;
        for (int k = 0; k < bp.n_red; k++) {
            L.red_bc.push_back((int32_t)b);
            L.red_chunk.push_back(k);
        }
        const int na = std::max(1, (bp.n_links + BC_CHUNK - 1) / BC_CHUNK);
        for (int k = 0; k < na; k++) {
            L.app_bc.push_back((int32_t)b);
            L.app_chunk.push_back(k);
        }
    }
    // immersed boundary: band = fluid cells within 3 cells (kernel support 2 +
    // one cell of wall travel) of any reference position
    for (int q = 0; q < ni; q++) {
        const lbm_instance_desc &d = cfg->inst[q];
        InstParam &ip = L.inst[q];
        ip.ib_off = (int)L.ib_dA.size();
        ip.n_ib = (int)d.n_ib;
        if (d.n_ib <= 0) continue;
        {
            // filaments: global node indices; interior nodes that are not
            // pinned are moved by the filament kernel (pinned code 2)
            int64_t o = 0;
            for (int64_t k = 0; k < d.ib_n_fil; k++) {
                const int64_t c = d.ib_fil_count[k];
                L.fil_start.push_back((int32_t)L.fil_nodes.size());
                L.fil_count.push_back((int32_t)c);
                for (int a = 0; a < 3; a++) L.fil_par.push_back(d.ib_fil_par[3 * k + a]);
                for (int64_t i = 0; i < c; i++) L.fil_nodes.push_back((int32_t)(ip.ib_off + d.ib_fil_nodes[o + i]));
                L.max_fil = std::max(L.max_fil, (int)c);
                o += c;
            }
        }
        const int nx = d.nx, ny = d.ny, nz = d.nz;
        for (int64_t s = 0; s < d.n_ib; s++) {
            for (int a = 0; a < 3; a++) L.ib_X0.push_back(d.ib_X0[3 * s + a]);
            L.ib_dA.push_back(d.ib_dA[s]);
            L.ib_ks.push_back(d.ib_ks[s]);
            L.ib_pinned.push_back(d.ib_pinned[s] ? 1 : 0);
            int i0[3];
            for (int a = 0; a < 3; a++) i0[a] = (int)std::floor(d.ib_X0[3 * s + a] - 0.5);
            for (int a = 0; a < 3; a++) L.ib_ref.push_back(i0[a]);
            for (int a = 0; a < 3; a++) L.ib_g0.push_back((float)((d.ib_X0[3 * s + a] - 0.5) - i0[a]));
            uint64_t mask[4] = {0, 0, 0, 0};
            for (int jz = 0; jz < 6; jz++)
                for (int jy = 0; jy < 6; jy++) {
                    const int y = i0[1] - 2 + jy, z = i0[2] - 2 + jz;
                    int32_t base = 0;
                    if (y >= 0 && y < ny && z >= 0 && z < nz) {
                        const int r = L.rowid[ip.rowid_off + y + ny * z];
                        if (r >= 0) {
                            const RowInfo &ri = L.rows[r];
                            base = ri.off - ri.x0;
                            for (int jx = 0; jx < 6; jx++) {
                                const int x = i0[0] - 2 + jx;
                                if (x < ri.x0 || x >= ri.x0 + ri.len) continue;
                                if (d.node[x + (int64_t)nx * (y + (int64_t)ny * z)] != 0) continue;
                                const int bit = jx + 6 * (jy + 6 * jz);
                                mask[bit >> 6] |= 1ull << (bit & 63);
                            }
                        }
                    }
                    L.ib_lines.push_back(base);
                }
            for (int k = 0; k < 4; k++) L.ib_mask.push_back(mask[k]);
            for (int dz = -2; dz <= 3; dz++)
                for (int dy = -2; dy <= 3; dy++)
                    for (int dx = -2; dx <= 3; dx++) {
                        int x = i0[0] + dx, y = i0[1] + dy, z = i0[2] + dz;
                        if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                        int64_t b = x + (int64_t)nx * (y + (int64_t)ny * z);
                        if (d.node[b] != 0) continue;
                        int r = L.rowid[ip.rowid_off + y + ny * z];
                        int64_t c = L.rows[r].off + (x - L.rows[r].x0);
                        L.flags[c] |= FL_BAND;
                    }
        }
    }
    for (int64_t c = 0; c < L.n_stored; c++)
        if (L.flags[c] & FL_BAND) L.band.push_back((int32_t)c);
    for (size_t k = 0; k < L.fil_start.size(); k++)
        for (int i = 1; i + 1 < L.fil_count[k]; i++) {
            uint8_t &pin = L.ib_pinned[L.fil_nodes[L.fil_start[k] + i]];
            if (pin == 0) pin = 2;
        }
    return "";
}

// Slabs of the pipelined step with wall nodes.  The compact cells are cut at
// the first row of lattice planes z = 0, 4, 8, ... of an instance, about
// n_stored / want cells apart, so that within an instance two cuts are at
// least 4 planes apart.  A wall node belongs to the slab of its reference
// plane; its kernel support (the 6^3 box around the reference cell, planes
// z_ref - 2 .. z_ref + 3) then lies in its own slab and the two next to it,
// and a pull reaches one plane, so:
//   * the band velocities of slab s read populations of slabs s-1 .. s+1;
//   * the node kernel of slab s gathers and spreads only in slabs s-1 .. s+1;
//   * stream-collide of slab s needs the spreading of slabs s-1 .. s+1.
// The second of these is checked here for every node against its support
// table; if it failed the tables stay empty (serial step).  Filaments couple
// nodes along the whole vessel, so they keep the serial step.
void build_slabs(Layout &L, int want) {
    L.slab_cell.clear();
    L.slab_band.clear();
    L.slab_node.clear();
    L.node_order.clear();
    const int64_t ns = (int64_t)L.ib_dA.size();
    if (want < 3 || ns == 0 || !L.fil_start.empty() || L.n_stored == 0) return;
    const int64_t target = std::max<int64_t>(1, L.n_stored / want);
    std::vector<int32_t> cut = {0};
    const size_t nrow = L.rows.size() - 1;  // without the sentinel
    for (size_t r = 1; r < nrow; r++) {
        const RowInfo &ri = L.rows[r], &rp = L.rows[r - 1];
        const bool plane_start = rp.z != ri.z || rp.inst != ri.inst;
        if (!plane_start || (ri.z % 4) != 0) continue;
        if ((int64_t)ri.off - cut.back() >= target) cut.push_back(ri.off);
    }
    cut.push_back((int32_t)L.n_stored);
    const int K = (int)cut.size() - 1;
    if (K < 3) return;
    auto slab_of_cell = [&](int64_t c) {
        return (int)(std::upper_bound(cut.begin(), cut.end(), (int32_t)c) - cut.begin()) - 1;
    };
    // slab of every plane of every instance: that of its first stored row, or
    // of the nearest plane above with rows
    std::vector<std::vector<int>> plane_slab(L.inst.size());
    for (size_t q = 0; q < L.inst.size(); q++) plane_slab[q].assign((size_t)std::max(1, L.inst[q].nz), -1);
    for (size_t r = 0; r < nrow; r++) {
        const RowInfo &ri = L.rows[r];
        int &ps = plane_slab[ri.inst][ri.z];
        if (ps < 0) ps = slab_of_cell(ri.off);
    }
    for (size_t q = 0; q < L.inst.size(); q++) {
        auto &v = plane_slab[q];
        int next = K - 1;
        for (int z = (int)v.size() - 1; z >= 0; z--) {
            if (v[z] < 0) v[z] = next;
            next = v[z];
        }
    }
    std::vector<int> node_slab((size_t)ns);
    std::vector<int64_t> per(K + 1, 0);
    size_t node0 = 0;
    for (size_t q = 0; q < L.inst.size(); q++) {
        const InstParam &ip = L.inst[q];
        for (int k = 0; k < ip.n_ib; k++) {
            const size_t s = node0 + k;
            const int z = std::min(std::max(L.ib_ref[3 * s + 2], 0), ip.nz - 1);
            const int sl = plane_slab[q][z];
            // every stored cell of the support box must lie in slabs sl - 1 .. sl + 1
            for (int j = 0; j < 36; j++) {
                const int64_t base = L.ib_lines[36 * s + j];
                for (int jx = 0; jx < 6; jx++) {
                    const int bit = jx + 6 * j;
                    if (!((L.ib_mask[4 * s + (bit >> 6)] >> (bit & 63)) & 1ull)) continue;
                    const int cs = slab_of_cell(base + L.ib_ref[3 * s] - 2 + jx);
                    if (cs < sl - 1 || cs > sl + 1) return;  // keep the serial step
                }
            }
            node_slab[s] = sl;
            per[sl + 1]++;
        }
        node0 += (size_t)ip.n_ib;
    }
    for (int k = 0; k < K; k++) per[k + 1] += per[k];
    L.node_order.assign((size_t)ns, 0);
    std::vector<int64_t> fill(per.begin(), per.end() - 1);
    for (int64_t s = 0; s < ns; s++) L.node_order[fill[node_slab[s]]++] = (int32_t)s;  // stable within a slab
    L.slab_cell = cut;
    for (int k = 0; k <= K; k++) {
        L.slab_node.push_back((int32_t)per[k]);
        L.slab_band.push_back((int32_t)(std::lower_bound(L.band.begin(), L.band.end(), cut[k]) - L.band.begin()));
    }
}

}  // namespace lbm
