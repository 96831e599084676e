// Fused stream-collide kernel (one launch per time step over every stored
// cell of every instance) and its launcher with the autotuner's variants.
#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Fused stream-collide.  For each fluid cell x and direction i the pulled
// population is f*_i(x - e_i) (or f*_opp(i)(x) when x - e_i is a rigid wall:
// halfway bounce-back).  Then P = c_s^2 sum f, j = sum e f, v = j + b/2
// (Eqs. rho, v), f^eq (Eq. feq), the forcing F_i (Eq. f) and BGK relaxation
// (Eq. fi).  With s = f - w: sum f = 1 + sum s, j = sum e s, and
// f^eq_i - w_i = w_i (sum s + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2).
// Occupancy request to ptxas (template parameter MINB: at least MINB resident
// 256-thread blocks per SM).  MINB = 6 caps the kernel at 40 registers (75 %
// occupancy) without spills; on the aorta it ran at 121 us per launch vs
// 131 us at 48 registers (5 blocks) and 129 us at 32 registers (8 blocks,
// with spills).  CPT > 1 gives each thread CPT independent cells, one grid
// stride apart, whose loads are all issued before any of them is consumed
// (more bytes in flight per thread at a lower occupancy).  The variants are
// kept for the run-time autotuner.  desc = 1 maps the blocks to the cells in
// descending order, so that a launch starts on the lines the previous kernel
// touched last (still in L2).
template <class S, int MINB, int CPT>
__global__ void __launch_bounds__(256, MINB)
    k_stream_collide(const S *__restrict__ fin, S *__restrict__ fout, KParams p, int desc) {
    using R = typename Storage<S>::R;
    const int bid = desc ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int t = bid * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (t == 0 && p.step) *p.step += 1;  // the step index t_n seen by the boundary kernels
    // population i of cell k lives at fin[pidx(i, k, N)]; 19 N < 2^31 is checked at creation
    const uint32_t N = (uint32_t)p.n;
    R f[CPT][NQ];
    R om[CPT];
    uint32_t fl[CPT];
#pragma unroll
    for (int u = 0; u < CPT; u++) {
        const int c = t + u * stride;
        fl[u] = c < p.n ? __ldg(&p.flags[c]) : 0u;
        om[u] = R(0);
        if (!(fl[u] & FL_ACTIVE)) continue;
        const int r = find_row(p, c);
        om[u] = omega_of<R>(p, __ldg(&p.rows[r].inst));
        const int x = __ldg(&p.rows[r].x0) + (c - __ldg(&p.rows[r].off));
        const int *nb = p.rows[r].nb;
#pragma unroll
        for (int i = 0; i < NQ; i++) {
            uint32_t off;
            if (i == 0) off = pidx(0, (uint32_t)c, N);
            else if (fl[u] & (1u << i)) off = pidx(opp(i), (uint32_t)c, N);
            else if (nbk(i) == 4) off = pidx(i, (uint32_t)(c - cx(i)), N);  // along x: the own row, no table
            else off = pidx(i, (uint32_t)(__ldg(&nb[nbk(i)]) + x - cx(i)), N);
            f[u][i] = Storage<S>::ld(fin + off);
        }
    }
#pragma unroll
    for (int u = 0; u < CPT; u++) {
        if (!(fl[u] & FL_ACTIVE)) continue;
        const int c = t + u * stride;
        R sd = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < NQ; i++) {
            sd += f[u][i];
            if (cx(i)) jx += cx(i) * f[u][i];
            if (cy(i)) jy += cy(i) * f[u][i];
            if (cz(i)) jz += cz(i) * f[u][i];
        }
        R bx = 0, by = 0, bz = 0;
        const bool band = (fl[u] & FL_BAND) != 0;
        if (band) {
            const typename Vec4<R>::T bb = static_cast<const typename Vec4<R>::T *>(p.b)[c];
            bx = bb.x;
            by = bb.y;
            bz = bb.z;
        }
        const R vx = jx + R(0.5) * bx, vy = jy + R(0.5) * by, vz = jz + R(0.5) * bz;
        if (fl[u] & FL_XF) {
            R *aux = static_cast<R *>(p.aux);
            aux[c] = sd;
            aux[N + c] = jx;
            aux[2 * N + c] = jy;
            aux[3 * N + c] = jz;
        }
        const R vv = vx * vx + vy * vy + vz * vz;
        if (!(sd - sd == R(0)) || !(vv <= R(0.09))) atomicOr(p.status, 1u);

        const R omega = om[u];
        const R usq = R(1.5) * vv;
        const R kf = R(1) - R(0.5) * omega;
#pragma unroll
        for (int i = 0; i < NQ; i++) {
            const R w = (R)wgt(i);
            const R eu = R(cx(i)) * vx + R(cy(i)) * vy + R(cz(i)) * vz;
            const R seq = w * (sd + R(3) * eu + R(4.5) * eu * eu - usq);
            R post = f[u][i] - omega * (f[u][i] - seq);
            if (band) {
                const R eb = R(cx(i)) * bx + R(cy(i)) * by + R(cz(i)) * bz;
                const R vb = vx * bx + vy * by + vz * bz;
                post += kf * w * (R(3) * (eb - vb) + R(9) * eu * eb);
            }
            Storage<S>::st(fout + pidx(i, (uint32_t)c, N), post);
        }
    }
}

// ---------------------------------------------------------------------------
// launcher

// variants: {min blocks per SM, cells per thread}
static const int kVariants[SC_VARIANTS][2] = {{6, 1}, {8, 1}, {5, 1}, {4, 2}, {3, 2}};

int stream_collide_min_blocks(int variant) { return kVariants[variant][0]; }
int stream_collide_cells_per_thread(int variant) { return kVariants[variant][1]; }

cudaError_t launch_stream_collide(int prec, const void *fin, void *fout, const KParams &p, int block,
                                  int variant, cudaStream_t s, int desc) {
    if (p.n == 0) return cudaSuccess;
    const int cpt = kVariants[variant][1];
    const int grid = (int)((p.n + (long long)block * cpt - 1) / ((long long)block * cpt));
    switch (variant) {
    case 1:
        DISPATCH(prec, (k_stream_collide<S, 8, 1><<<grid, block, 0, s>>>(static_cast<const S *>(fin), as<S>(fout), p, desc)));
        break;
    case 2:
        DISPATCH(prec, (k_stream_collide<S, 5, 1><<<grid, block, 0, s>>>(static_cast<const S *>(fin), as<S>(fout), p, desc)));
        break;
    case 3:
        DISPATCH(prec, (k_stream_collide<S, 4, 2><<<grid, block, 0, s>>>(static_cast<const S *>(fin), as<S>(fout), p, desc)));
        break;
    case 4:
        DISPATCH(prec, (k_stream_collide<S, 3, 2><<<grid, block, 0, s>>>(static_cast<const S *>(fin), as<S>(fout), p, desc)));
        break;
    default:
        DISPATCH(prec, (k_stream_collide<S, 6, 1><<<grid, block, 0, s>>>(static_cast<const S *>(fin), as<S>(fout), p, desc)));
        break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
