// Immersed-boundary exchange between Lagrangian wall nodes and the lattice
// (Section 2.3.2, Eqs. LagForce, interpolation, EulForce) and the wall-node
// update (linear springs to the reference position, symplectic Euler).
//
//   k_band_moments  unforced velocity j/rho0 of f(t_n) at every band cell
//                   (the cells within the support of a wall node) and b = 0
//   k_ib_nodes      one thread per wall node: interpolate V_f with the 4-point
//                   cosine delta, update the penalty integral and the force
//                   F = alpha I + beta (V_f - V_s) on the fluid, spread
//                   F delta dA into b, then move the node.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_kernels.h"

namespace lbm {

template <class S> struct IbStorage;
template <> struct IbStorage<float> { using R = float; static __device__ float ld(const float *p) { return __ldg(p); } };
template <> struct IbStorage<double> { using R = double; static __device__ double ld(const double *p) { return __ldg(p); } };
template <> struct IbStorage<__half> { using R = float; static __device__ float ld(const __half *p) { return __half2float(__ldg(p)); } };
template <> struct IbStorage<__nv_bfloat16> {
    using R = float;
    static __device__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
};

template <class S>
__global__ void k_band_moments(const S *__restrict__ fin, KParams p, IbKParams ib) {
    using R = typename IbStorage<S>::R;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ib.n_band) return;
    const int c = ib.band[t];
    const uint32_t fl = p.flags[c];
    const size_t N = (size_t)p.n;
    int r = p.chunk_row[c >> 5];
    while (p.rows[r + 1].off <= c) r++;
    const int x = p.rows[r].x0 + (c - p.rows[r].off);
    R jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 1; i < NQ; i++) {
        size_t idx;
        if (fl & (1u << i)) idx = (size_t)opp(i) * N + c;
        else idx = (size_t)i * N + (size_t)(p.rows[r].nb[nbk(i)] + x - cx(i));
        const R fi = IbStorage<S>::ld(fin + idx);
        if (cx(i)) jx += cx(i) * fi;
        if (cy(i)) jy += cy(i) * fi;
        if (cz(i)) jz += cz(i) * fi;
    }
    R *v = static_cast<R *>(ib.vband);
    v[c] = jx;
    v[N + c] = jy;
    v[2 * N + c] = jz;
    R *b = static_cast<R *>(const_cast<void *>(p.b));
    b[c] = 0;
    b[N + c] = 0;
    b[2 * N + c] = 0;
}

// 4-point cosine discrete delta along one axis
__device__ __forceinline__ double phi(double r) {
    const double a = fabs(r);
    if (a >= 2.0) return 0.0;
    return 0.25 * (1.0 + cos(M_PI * r / 2.0));
}

template <class R> __device__ __forceinline__ void atomic_add(R *a, R v) { atomicAdd(a, v); }

template <class S>
__global__ void k_ib_nodes(KParams p, IbKParams ib) {
    using R = typename IbStorage<S>::R;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ib.n_nodes) return;
    const InstParam ip = ib.inst[ib.node_inst[s]];
    const size_t N = (size_t)p.n;
    double X[3], Vs[3];
    int i0[3];
    double ph[3][4];
    for (int a = 0; a < 3; a++) {
        X[a] = ib.X[3 * s + a];
        Vs[a] = ib.Vs[3 * s + a];
        i0[a] = (int)floor(X[a] - 0.5);
        for (int k = 0; k < 4; k++) ph[a][k] = phi((double)(i0[a] + k - 1) + 0.5 - X[a]);
    }
    const int dims[3] = {ip.nx, ip.ny, ip.nz};
    int cell[64];
    const R *vb = static_cast<const R *>(ib.vband);
    double Vf[3] = {0.0, 0.0, 0.0};
    bool out_of_band = false;
    for (int dz = 0; dz < 4; dz++)
        for (int dy = 0; dy < 4; dy++)
            for (int dx = 0; dx < 4; dx++) {
                const int k = dx + 4 * (dy + 4 * dz);
                cell[k] = -1;
                const int x = i0[0] + dx - 1, y = i0[1] + dy - 1, z = i0[2] + dz - 1;
                if (x < 0 || x >= dims[0] || y < 0 || y >= dims[1] || z < 0 || z >= dims[2]) continue;
                const int r = ib.rowid[ip.rowid_off + y + ip.ny * z];
                if (r < 0) continue;
                const int x0 = p.rows[r].x0, len = p.rows[r].len;
                if (x < x0 || x >= x0 + len) continue;
                const int c = p.rows[r].off + (x - x0);
                const uint32_t fl = p.flags[c];
                if (!(fl & FL_ACTIVE)) continue;
                if (!(fl & FL_BAND)) {
                    out_of_band = true;
                    continue;
                }
                cell[k] = c;
                const double d = ph[0][dx] * ph[1][dy] * ph[2][dz];
                Vf[0] += (double)vb[c] * d;
                Vf[1] += (double)vb[N + c] * d;
                Vf[2] += (double)vb[2 * N + c] * d;
            }
    if (out_of_band) atomicOr(p.status, 2u);
    double F[3];
    for (int a = 0; a < 3; a++) {
        const double dv = Vf[a] - Vs[a];
        const double I = ib.I[3 * s + a] + dv;
        ib.I[3 * s + a] = I;
        F[a] = ip.alpha * I + ip.beta * dv;
        ib.F[3 * s + a] = F[a];
        ib.Vf[3 * s + a] = Vf[a];
    }
    R *b = static_cast<R *>(const_cast<void *>(p.b));
    const double dA = ib.dA[s];
    for (int dz = 0; dz < 4; dz++)
        for (int dy = 0; dy < 4; dy++)
            for (int dx = 0; dx < 4; dx++) {
                const int c = cell[dx + 4 * (dy + 4 * dz)];
                if (c < 0) continue;
                const double d = ph[0][dx] * ph[1][dy] * ph[2][dz] * dA;
                atomic_add<R>(&b[c], (R)(F[0] * d));
                atomic_add<R>(&b[N + c], (R)(F[1] * d));
                atomic_add<R>(&b[2 * N + c], (R)(F[2] * d));
            }
    if (!ib.pinned[s]) {
        for (int a = 0; a < 3; a++) {
            const double acc = (-ib.ks[s] * (X[a] - ib.X0[3 * s + a]) - F[a]) / ip.ms;
            const double v = Vs[a] + acc;
            ib.Vs[3 * s + a] = v;
            ib.X[3 * s + a] = X[a] + v;
        }
    }
}

cudaError_t launch_ib(int prec, const void *fin, const KParams &p, const IbKParams &ib, cudaStream_t st) {
    if (ib.n_nodes == 0) return cudaSuccess;
    const int block = 256;
    const int gb = (ib.n_band + block - 1) / block;
    const int gn = (ib.n_nodes + block - 1) / block;
    switch (prec) {
    case 0:
        if (gb) k_band_moments<float><<<gb, block, 0, st>>>(static_cast<const float *>(fin), p, ib);
        k_ib_nodes<float><<<gn, block, 0, st>>>(p, ib);
        break;
    case 1:
        if (gb) k_band_moments<__half><<<gb, block, 0, st>>>(static_cast<const __half *>(fin), p, ib);
        k_ib_nodes<__half><<<gn, block, 0, st>>>(p, ib);
        break;
    case 2:
        if (gb) k_band_moments<__nv_bfloat16><<<gb, block, 0, st>>>(static_cast<const __nv_bfloat16 *>(fin), p, ib);
        k_ib_nodes<__nv_bfloat16><<<gn, block, 0, st>>>(p, ib);
        break;
    default:
        if (gb) k_band_moments<double><<<gb, block, 0, st>>>(static_cast<const double *>(fin), p, ib);
        k_ib_nodes<double><<<gn, block, 0, st>>>(p, ib);
        break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
