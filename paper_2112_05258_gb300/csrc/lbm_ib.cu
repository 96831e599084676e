// Immersed-boundary exchange between Lagrangian wall nodes and the lattice
// (Section 2.3.2, Eqs. LagForce, interpolation, EulForce) and the wall-node
// update (linear springs to the reference position, symplectic Euler).
//
//   k_band_moments  fluid velocity j/rho0 + b/2 of f(t_n) at every band cell
//                   (the cells within reach of a wall node's kernel support),
//                   b being the force density of the previous step, and then
//                   b = 0 there; both as one 4-vector per cell
//   k_ib_nodes      1, 2 or 4 threads per wall node: gather V_f over the 64
//                   support cells of the 4-point cosine delta, penalty
//                   integral and force F = alpha I + beta (V_f - V_s) on the
//                   fluid, spreading of F delta dA with one vector atomic per
//                   cell, spring update.  With FP32 arithmetic (FP32, FP16 or
//                   BF16 storage) the node state is FP32 and the position is
//                   kept as the displacement D = X - X0 (|D| < 1 cell, so its
//                   rounding is ~6e-8 cells where X itself would round to
//                   ~6e-5 at x ~ 1000); FP64 storage keeps the FP64 state.
//   k_filament      one CTA per filament of wall nodes: SGFD tension and
//                   bending forces (Section 2.3.2) at X(t_n) from shared
//                   memory, then the wall update of its interior nodes.
#include "lbm_device.cuh"

namespace lbm {

// Entries [t0, t1) of the band list (ascending cells).  Blocks take them in
// descending cell order: stream-collide finished on the highest cells, whose
// lines are still in L2.
template <class S>
__global__ void k_band_moments(const S *__restrict__ fin, KParams p, IbKParams ib, int t0, int t1) {
    using R = typename Storage<S>::R;
    using V = typename Vec4<R>::T;
    const int t = t0 + (int)(gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= t1) return;
    const int c = ib.band[t];
    const uint32_t fl = p.flags[c];
    const size_t N = (size_t)p.n;
    const int2 ch = reinterpret_cast<const int2 *>(p.chunk_row)[c >> 5];
    const int r = ch.x + __popc((uint32_t)ch.y & ((2u << (c & 31)) - 1u));
    const int x = p.rows[r].x0 + (c - p.rows[r].off);
    R jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 1; i < NQ; i++) {
        size_t idx;
        if (fl & (1u << i)) idx = pidx(opp(i), (uint32_t)c, (uint32_t)N);
        else if (nbk(i) == 4) idx = pidx(i, (uint32_t)(c - cx(i)), (uint32_t)N);  // along x: the own row
        else idx = pidx(i, (uint32_t)(p.rows[r].nb[nbk(i)] + x - cx(i)), (uint32_t)N);
        const R fi = Storage<S>::ld(fin + idx);
        if (cx(i)) jx += cx(i) * fi;
        if (cy(i)) jy += cy(i) * fi;
        if (cz(i)) jz += cz(i) * fi;
    }
    // fluid velocity of Eq. v with the force density of the previous step,
    // which is then cleared for this step's spreading
    V *b = static_cast<V *>(const_cast<void *>(p.b));
    const V bo = b[c];
    V v;
    v.x = jx + R(0.5) * bo.x;
    v.y = jy + R(0.5) * bo.y;
    v.z = jz + R(0.5) * bo.z;
    v.w = 0;
    static_cast<V *>(ib.vband)[c] = v;
    V z;
    z.x = z.y = z.z = z.w = 0;
    b[c] = z;
}

// Weights of the 4-point cosine delta phi(r) = (1 + cos(pi r / 2)) / 4 at the
// offsets r_k = (k - 1) - th, k = 0..3, th in [0, 1): with C = cos(pi th / 2)
// and S = sin(pi th / 2) they are (1 - S)/4, (1 + C)/4, (1 + S)/4, (1 - C)/4.
template <class R> __device__ __forceinline__ R delta_weight(R Sn, R Cs, int k) {
    const R v = (k == 0) ? -Sn : (k == 1) ? Cs : (k == 2) ? Sn : -Cs;
    return R(0.25) * (R(1) + v);
}
__device__ __forceinline__ void sincospi_half(float th, float *s, float *c) { sincospif(0.5f * th, s, c); }
__device__ __forceinline__ void sincospi_half(double th, double *s, double *c) { sincospi(0.5 * th, s, c); }

__device__ __forceinline__ void vec_atomic_add(float4 *a, float4 v) { atomicAdd(a, v); }
__device__ __forceinline__ void vec_atomic_add(double4a *a, double4a v) {
    atomicAdd(&a->x, v.x);
    atomicAdd(&a->y, v.y);
    atomicAdd(&a->z, v.z);
}

// TPN threads per wall node (1, 2 or 4); lane q of a node's group owns the
// support planes dz = q * PL .. q * PL + PL - 1 (PL = 4 / TPN) of the 4-point
// cosine delta.  The lattice lines and fluid cells of the support come from
// the node's precomputed table (no row lookup, no flag loads), and the line
// bases and a mask of the valid support cells stay in registers for the
// spreading pass.  A warp holds 32 / TPN consecutive nodes
// of a ring.  The group's partial velocities are summed with butterfly
// shuffles, which every lane evaluates in the same order, so all lanes
// compute the same penalty force; lane 0 writes the node state.
// The kernel takes the wall nodes ib.order[k0 .. k1) (all nodes in index
// order when ib.order is null).
//
// With two or four threads per node, consecutive nodes (the pair k0 + 2m, k0 + 2m + 1,
// neighbours on a ring, whose supports share about 70 % of their cells) merge
// their spreading: the first node of the pair adds the second node's
// contribution F' delta(x - X') dA' to every cell of its own support that
// the second support also covers (one vector atomic for both), and the second
// node spreads only into the cells outside the first one's support.  On the
// aorta membrane this takes the atomics from 64 to about 42 per node.  The
// partner's weights, reference cell and force come by shuffles within the
// pair's lanes; a pair whose supports do not overlap, or with a node out
// of its band or past k1, spreads node by node.
template <class S, int TPN>
__global__ void __launch_bounds__(128) k_ib_nodes(KParams p, IbKParams ib, int k0, int k1) {
    using R = typename Storage<S>::R;
    using V = typename Vec4<R>::T;
    constexpr int PL = 4 / TPN;
    constexpr bool PAIRED = TPN >= 2;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int kk = k0 + gt / TPN, q = gt % TPN;
    // the lanes of a node leave together; with pairs, those of a pair (a
    // second node past k1 stays, idle, for the pair's shuffles)
    if ((PAIRED ? k0 + ((gt / TPN) & ~1) : kk) >= k1) return;
    const bool dead = kk >= k1;
    const int s = ib.order ? ib.order[dead ? k1 - 1 : kk] : (dead ? k1 - 1 : kk);
    constexpr bool F32 = sizeof(R) == 4;  // FP32 node state (displacements)
    if (q == 0) {  // lane 0 reads the node state after the gathers: bring it towards L2 meanwhile
        if (F32) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.Vs32 + 3 * s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.I32 + 3 * s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.ks32 + s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.dA32 + s));
        } else {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.Vs + 3 * s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.I + 3 * s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.X0 + 3 * s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.ks + s));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.dA + s));
        }
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.pinned + s));
    }
    // the support-line table (36 entries) and the fluid mask are read once
    // the node's cell is known
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.lines + 36 * (size_t)s + (36 / TPN) * q));
    if (q == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(ib.mask + 4 * (size_t)s));
    const InstParam &ip = ib.inst[ib.node_inst[s]];
    // X - 1/2 = i0 + th with th in [0, 1): i0 = ref + d, where d is the cell
    // offset from the reference cell ref = floor(X0 - 1/2)
    double X[3];
    float D[3];
    int i0[3], d[3];
    R w[3][4];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R th;
        if (F32) {
            D[a] = ib.D32[3 * s + a];
            const float t = ib.g0[3 * s + a] + D[a];  // X - 1/2 - ref
            const float ft = floorf(t);
            d[a] = (int)ft;
            th = (R)(t - ft);
        } else {
            X[a] = ib.X[3 * s + a];
            const double h = X[a] - 0.5;
            const double fl0 = floor(h);
            d[a] = (int)fl0 - ib.ref[3 * s + a];
            th = (R)(h - fl0);
        }
        i0[a] = ib.ref[3 * s + a] + d[a];
        R Sn, Cs;
        sincospi_half(th, &Sn, &Cs);
#pragma unroll
        for (int k = 0; k < 4; k++) w[a][k] = delta_weight<R>(Sn, Cs, k);
    }
    // support cells through the node's precomputed line table and fluid mask
    // (box of 6^3 cells around its reference cell; the node may move by less
    // than one cell from it, else the status word reports it)
    bool out_of_band = false;
#pragma unroll
    for (int a = 0; a < 3; a++) out_of_band |= (d[a] < -1 || d[a] > 1);
    const V *vb = static_cast<const V *>(ib.vband);
    R vx = 0, vy = 0, vz = 0;
    int lb[4 * PL];
    uint64_t valid = 0;  // bit dx + 4 (dy + 4 j) for the lane's plane j
    if (!out_of_band) {
        const int32_t *lines = ib.lines + 36 * (size_t)s;
        const uint64_t m0 = ib.mask[4 * (size_t)s], m1 = ib.mask[4 * (size_t)s + 1];
        const uint64_t m2 = ib.mask[4 * (size_t)s + 2], m3 = ib.mask[4 * (size_t)s + 3];
#pragma unroll
        for (int j = 0; j < PL; j++) {
            const int dz = q * PL + j;
            const int jz = d[2] + dz + 1;
            const R wz = w[2][0] * (dz == 0) + w[2][1] * (dz == 1) + w[2][2] * (dz == 2) + w[2][3] * (dz == 3);
#pragma unroll
            for (int dy = 0; dy < 4; dy++) {
                const int jy = d[1] + dy + 1;
                const int base = lines[jy + 6 * jz];
                lb[dy + 4 * j] = base;
                const R wyz = w[1][dy] * wz;
#pragma unroll
                for (int dx = 0; dx < 4; dx++) {
                    const int bit = d[0] + dx + 1 + 6 * (jy + 6 * jz);
                    const uint64_t word = bit < 64 ? m0 : bit < 128 ? m1 : bit < 192 ? m2 : m3;
                    const bool ok = (word >> (bit & 63)) & 1ull;  // else a wall or boundary slot: no fluid
                    valid |= (uint64_t)ok << (dx + 4 * (dy + 4 * j));
                    // branch-free, so that the loads can all be in flight: a
                    // missing cell reads slot 0 (zeroed at creation, finite)
                    // with weight 0
                    const V v = vb[ok ? base + i0[0] + dx - 1 : 0];
                    const R dd = ok ? w[0][dx] * wyz : R(0);
                    vx += v.x * dd;
                    vy += v.y * dd;
                    vz += v.z * dd;
                }
            }
        }
    }
    if (out_of_band && !dead) atomicOr(p.status, 2u);
    if (dead) valid = 0;
    const unsigned grp = TPN > 1 ? ((1u << TPN) - 1u) << ((threadIdx.x & 31) & ~(TPN - 1)) : 0u;
    if (TPN > 1) {
#pragma unroll
        for (int o = 1; o < TPN; o <<= 1) {
            vx += __shfl_xor_sync(grp, vx, o, TPN);
            vy += __shfl_xor_sync(grp, vy, o, TPN);
            vz += __shfl_xor_sync(grp, vz, o, TPN);
        }
    }
    // the penalty force on lane 0 of the node's group (in the node state's
    // precision), which then hands F dA to the other lanes for their planes
    // of the spreading
    double F[3], Vs[3];
    float F32v[3], Vs32v[3];
    R Fx = 0, Fy = 0, Fz = 0;
    if (q == 0 && !dead) {
        if (F32) {
            const float Vf[3] = {(float)vx, (float)vy, (float)vz};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                Vs32v[a] = ib.Vs32[3 * s + a];
                const float dv = Vf[a] - Vs32v[a];
                const float I = ib.I32[3 * s + a] + dv;
                F32v[a] = ip.alpha_f * I + ip.beta_f * dv;
                ib.I32[3 * s + a] = I;
                ib.F32[3 * s + a] = F32v[a];
                ib.Vf32[3 * s + a] = Vf[a];
            }
            const R dA = (R)ib.dA32[s];
            Fx = (R)F32v[0] * dA;
            Fy = (R)F32v[1] * dA;
            Fz = (R)F32v[2] * dA;
        } else {
            const double Vf[3] = {(double)vx, (double)vy, (double)vz};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                Vs[a] = ib.Vs[3 * s + a];
                const double dv = Vf[a] - Vs[a];
                const double I = ib.I[3 * s + a] + dv;
                F[a] = ip.alpha * I + ip.beta * dv;
                ib.I[3 * s + a] = I;
                ib.F[3 * s + a] = F[a];
                ib.Vf[3 * s + a] = Vf[a];
            }
            const R dA = (R)ib.dA[s];
            Fx = (R)F[0] * dA;
            Fy = (R)F[1] * dA;
            Fz = (R)F[2] * dA;
        }
    }
    if (TPN > 1) {
        Fx = __shfl_sync(grp, Fx, 0, TPN);
        Fy = __shfl_sync(grp, Fy, 0, TPN);
        Fz = __shfl_sync(grp, Fz, 0, TPN);
    }
    // pair merge: the partner's offsets e = d - (i0' - i0) of this lane's
    // support cells d; pw[a][d] = partner weight at e (0 outside [0, 4)), and
    // pin[a] the bits d with e inside, per axis (z: this lane's planes)
    bool merge = false, first = true;
    R pw[3][4], pF[3] = {R(0), R(0), R(0)};
    uint32_t pin[3] = {0u, 0u, 0u};
    if (PAIRED) {
        const unsigned pm = ((1u << (2 * TPN)) - 1u) << ((threadIdx.x & 31) & ~(2u * TPN - 1u));  // the pair's lanes
        const bool ok = !dead && !out_of_band;
        first = ((gt / TPN) & 1) == 0;
        const bool pok = __shfl_xor_sync(pm, (int)ok, TPN) != 0;
        int D[3];
        bool near = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            D[a] = __shfl_xor_sync(pm, i0[a], TPN) - i0[a];
            near = near && D[a] > -4 && D[a] < 4;
        }
        R ow[3][4];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int k = 0; k < 4; k++) ow[a][k] = __shfl_xor_sync(pm, w[a][k], TPN);
        pF[0] = __shfl_xor_sync(pm, Fx, TPN);
        pF[1] = __shfl_xor_sync(pm, Fy, TPN);
        pF[2] = __shfl_xor_sync(pm, Fz, TPN);
        merge = ok && pok && near;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int dd = 0; dd < 4; dd++) {
                const int e = dd - D[a];
                R v = R(0);
#pragma unroll
                for (int k = 0; k < 4; k++) v = (e == k) ? ow[a][k] : v;
                pw[a][dd] = v;
                pin[a] |= (uint32_t)(e >= 0 && e < 4) << dd;
            }
    }
    V *b = static_cast<V *>(const_cast<void *>(p.b));
#pragma unroll
    for (int k = 0; k < 16 * PL; k++) {
        if (!((valid >> k) & 1ull)) continue;
        const int dx = k & 3, dy = (k >> 2) & 3, j = k >> 4;
        const int dz = q * PL + j;
        // the second node of a merged pair leaves the cells the first one covers
        if (PAIRED && merge && !first && ((pin[0] >> dx) & (pin[1] >> dy) & (pin[2] >> dz) & 1u)) continue;
        const R wz = w[2][0] * (dz == 0) + w[2][1] * (dz == 1) + w[2][2] * (dz == 2) + w[2][3] * (dz == 3);
        const int c = lb[dy + 4 * j] + i0[0] + dx - 1;
        const R d = w[0][dx] * (w[1][dy] * wz);
        V add;
        add.x = Fx * d;
        add.y = Fy * d;
        add.z = Fz * d;
        add.w = 0;
        if (PAIRED && merge && first) {
            const R pwz = pw[2][0] * (dz == 0) + pw[2][1] * (dz == 1) + pw[2][2] * (dz == 2) + pw[2][3] * (dz == 3);
            const R e = pw[0][dx] * (pw[1][dy] * pwz);
            add.x += pF[0] * e;
            add.y += pF[1] * e;
            add.z += pF[2] * e;
        }
        vec_atomic_add(&b[c], add);
    }
    if (q == 0 && !dead && ib.pinned[s] == 0) {  // pinned nodes stay; filament nodes move in k_filament
        if (F32) {
            const float ks = ib.ks32[s];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float acc = (-ks * D[a] - F32v[a]) * ip.inv_ms_f;
                const float v = Vs32v[a] + acc;
                ib.Vs32[3 * s + a] = v;
                ib.D32[3 * s + a] = D[a] + v;
            }
        } else {
            const double inv_ms = ip.inv_ms;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double acc = (-ib.ks[s] * (X[a] - ib.X0[3 * s + a]) - F[a]) * inv_ms;
                const double v = Vs[a] + acc;
                ib.Vs[3 * s + a] = v;
                ib.X[3 * s + a] = X[a] + v;
            }
        }
    }
}

// SGFD filament (Section 2.3.2): node i of a filament of n nodes at reference
// spacing ds, with simply supported ends (ghosts X_{-1} = 2 X_0 - X_1 and
// X_n = 2 X_{n-1} - X_{n-2}, so D+D- X vanishes at both ends):
//   T_{i+1/2} = Eh (|D0 X_{i+1/2}| - 1)                          (Eq. tension)
//   F_i = [(T D0 X)_{i+1/2} - (T D0 X)_{i-1/2}] / ds
//         - EI [K_{i+1} - 2 K_i + K_{i-1}] / ds^2,  K_j = D+D- X_j (Eq. bending)
// The filament's positions X(t_n) are staged in shared memory before any
// node moves, so every force sees the same time level; the interior nodes
// (pinned code 2) then take m_s dV/dt = -k_s (X - X0) + F_i - F_penalty
// with dt = 1 (V, then X), the central difference in time.
// FP64 division and square root are multi-instruction sequences on the
// FP64 pipe, which is narrow on this part: the kernel multiplies by 1/ds and
// 1/m_s, computed once per thread (one rounding more than dividing, far
// below the parity tolerance), and stages K_j and (T D0 X)_{j+1/2} once per
// node and segment in shared memory (one square root per segment).
constexpr int FIL_THREADS = 512;

template <bool F32>
__global__ void __launch_bounds__(FIL_THREADS) k_filament(KParams p, IbKParams ib) {
    extern __shared__ double sm[];
    const int k = blockIdx.x;
    const int n = ib.fil_count[k], st = ib.fil_start[k];
    double *P = sm;                 // X_{-1} .. X_n: P[3 (j + 1) + a] = X_j
    double *K = P + 3 * (n + 2);    // K_j = D+D- X_j, j = 0 .. n-1
    double *TD = K + 3 * n;         // (T D0 X)_{j+1/2}, j = 0 .. n-2
    const double ds = ib.fil_par[3 * k], Eh = ib.fil_par[3 * k + 1], EI = ib.fil_par[3 * k + 2];
    const double inv_ds = 1.0 / ds, inv_ds2 = inv_ds * inv_ds;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = ib.fil_nodes[st + i];
#pragma unroll
        for (int a = 0; a < 3; a++)
            P[3 * (i + 1) + a] = F32 ? ib.X0[3 * s + a] + (double)ib.D32[3 * s + a] : ib.X[3 * s + a];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        P[a] = 2.0 * P[3 + a] - P[6 + a];
        P[3 * (n + 1) + a] = 2.0 * P[3 * n + a] - P[3 * (n - 1) + a];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double *x = P + 3 * (j + 1);
#pragma unroll
        for (int a = 0; a < 3; a++) K[3 * j + a] = (x[3 + a] - 2.0 * x[a] + x[a - 3]) * inv_ds2;
        if (j + 1 < n) {
            double d[3], len2 = 0.0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                d[a] = (x[3 + a] - x[a]) * inv_ds;
                len2 += d[a] * d[a];
            }
            const double T = Eh * (sqrt(len2) - 1.0);
#pragma unroll
            for (int a = 0; a < 3; a++) TD[3 * j + a] = T * d[a];
        }
    }
    __syncthreads();
    for (int i = 1 + threadIdx.x; i < n - 1; i += blockDim.x) {
        const int s = ib.fil_nodes[st + i];
        if (ib.pinned[s] != 2) continue;
        const double inv_ms = ib.inst[ib.node_inst[s]].inv_ms;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double xa = P[3 * (i + 1) + a];
            const double ff = (TD[3 * i + a] - TD[3 * (i - 1) + a]) * inv_ds -
                              EI * (K[3 * (i + 1) + a] - 2.0 * K[3 * i + a] + K[3 * (i - 1) + a]) * inv_ds2;
            const double Fp = F32 ? (double)ib.F32[3 * s + a] : ib.F[3 * s + a];
            const double acc = (-ib.ks[s] * (xa - ib.X0[3 * s + a]) + ff - Fp) * inv_ms;
            if (F32) {
                const double v = (double)ib.Vs32[3 * s + a] + acc;
                ib.Vs32[3 * s + a] = (float)v;
                ib.D32[3 * s + a] = (float)((xa - ib.X0[3 * s + a]) + v);
            } else {
                const double v = ib.Vs[3 * s + a] + acc;
                ib.Vs[3 * s + a] = v;
                ib.X[3 * s + a] = xa + v;
            }
        }
    }
}

static size_t filament_smem(int max_fil) { return (size_t)(9 * max_fil + 6) * sizeof(double); }

cudaError_t prepare_filament_kernel(int max_fil) {
    cudaError_t e = cudaFuncSetAttribute(k_filament<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)filament_smem(max_fil));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_filament<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)filament_smem(max_fil));
    return e;
}

template <class S> static void launch_nodes(const KParams &p, const IbKParams &ib, int k0, int k1, cudaStream_t st) {
    const int tpn = ib.threads_per_node;
    const int grid = (int)(((long long)(k1 - k0) * tpn + 127) / 128);
    if (grid == 0) return;
    if (tpn == 1) k_ib_nodes<S, 1><<<grid, 128, 0, st>>>(p, ib, k0, k1);
    else if (tpn == 2) k_ib_nodes<S, 2><<<grid, 128, 0, st>>>(p, ib, k0, k1);
    else k_ib_nodes<S, 4><<<grid, 128, 0, st>>>(p, ib, k0, k1);
}

cudaError_t launch_band_moments(int prec, const void *fin, const KParams &p, const IbKParams &ib, int t0, int t1,
                                cudaStream_t st) {
    const int block = 256;
    const int gb = (t1 - t0 + block - 1) / block;
    if (gb <= 0) return cudaSuccess;
    DISPATCH(prec, (k_band_moments<S><<<gb, block, 0, st>>>(static_cast<const S *>(fin), p, ib, t0, t1)));
    return cudaGetLastError();
}

cudaError_t launch_ib_nodes(int prec, const KParams &p, const IbKParams &ib, int k0, int k1, cudaStream_t st) {
    DISPATCH(prec, (launch_nodes<S>(p, ib, k0, k1, st)));
    return cudaGetLastError();
}

cudaError_t launch_ib(int prec, const void *fin, const KParams &p, const IbKParams &ib, cudaStream_t st, bool band) {
    if (ib.n_nodes == 0) return cudaSuccess;
    cudaError_t e = band ? launch_band_moments(prec, fin, p, ib, 0, ib.n_band, st) : cudaSuccess;
    if (e == cudaSuccess) e = launch_ib_nodes(prec, p, ib, 0, ib.n_nodes, st);
    if (e == cudaSuccess && ib.n_fil) {
        if (prec == 3)
            k_filament<false><<<ib.n_fil, FIL_THREADS, filament_smem(ib.max_fil), st>>>(p, ib);
        else
            k_filament<true><<<ib.n_fil, FIL_THREADS, filament_smem(ib.max_fil), st>>>(p, ib);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace lbm
