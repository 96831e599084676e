// The 3D-axisymmetric D2Q9 lattice (Section 2.3.1, Eq. Afi) with the 0D
// boundaries of Section 2.2, and its C-ABI (include/lbm_axi.h).
//
//   k_axi_collide  one thread per node of the dense (x, r) grid: pull with
//                  halfway bounce-back and the mirror at the axis, moments,
//                  axisymmetric sources, Guo forcing, BGK collision
//   k_axi_gather   read-out of f(t_n) and of P, u_x, u_r
//   k_axi_init     inverse of the pull (lays out a given f(t_0))
//   k_axi_bc_reduce  FP64 area-weighted flow and pressure partial sums over
//                  chunks of every 0D boundary's first fluid layer
//   k_axi_bc_apply   per chunk of links: the 0D step from the partials and
//                  the ghost populations of Eq. Non-equilibrium3 (per node
//                  and per link in the compute type)
//
// Sources (derived from the axisymmetric incompressible equations, rho0 = 1;
// the printed h^(2) of Eq. AH1 is not legible): with j = sum e f (the
// unforced momentum), r = j_r-row + 1/2,
//   m   = -j_r / r,                 P = c_s^2 (sum f + m/2)
//   g_x = -(1 - 1/(2 tau)) Pi_xr / r - j_x j_r / r
//   g_r = -(1 - 1/(2 tau)) Pi_rr / r - 2 nu j_r / r^2 - j_r^2 / r
// where Pi = sum e e (f - f^eq(c_s^2 sum f, j)) is the non-equilibrium stress
// against the equilibrium of f's own moments (so that the isotropic part the
// mass source leaves in f's second moment does not enter the strain rate);
// v = j + g/2; the collision adds the Guo term of g and (1 - 1/(2 tau)) w_i m.
// Populations are stored as deviations s = f - w (FP32 or FP64), in SoA
// order f[i][j nx + x]; the resident state is f*(t_n) with the ghosts of
// t_{n+1} in the 0D boundary nodes' slots, as in the 3D lattice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm_axi.h"
#include "lbm_device.cuh"
#include "lbm_zero_d.cuh"

namespace lbm {
namespace axi {

constexpr int Q9 = 9;
__host__ __device__ constexpr int ex(int i) { return i == 1 || i == 5 || i == 7 ? 1 : (i == 2 || i == 6 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int er(int i) { return i == 3 || i == 5 || i == 8 ? 1 : (i == 4 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1); }
__host__ __device__ constexpr int mir(int i) {  // e_r -> -e_r
    return i == 3 ? 4 : i == 4 ? 3 : i == 5 ? 7 : i == 7 ? 5 : i == 6 ? 8 : i == 8 ? 6 : i;
}
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

enum : uint16_t { AF_FLUID = 1u << 9, AF_XF = 1u << 10 };  // bits 1..8: pull source is a wall

struct Params {
    int nx, nr;
    int n;                 // nx * nr
    const uint16_t *flags;
    void *aux;             // 6 x n compute type at first-layer nodes: s_sum + m/2, j_x, j_r, v_x, v_r, s_sum
    double tau;
    unsigned *status;
    // relaxation constants and 1/r per row in both arithmetic types (no
    // division or FP64 conversion per node): omega = 1/tau, k = 1 - 1/(2 tau),
    // nu = (tau - 1/2)/3
    float omega_f, k_f, nu_f;
    double omega_d, k_d, nu_d;
    const float *inv_r_f;
    const double *inv_r_d;
    long long *step;       // index t_n of the step in progress (advanced by the collide kernel)
};

template <class R> struct Consts;
template <> struct Consts<float> {
    static __device__ __forceinline__ void get(const Params &p, int j, float *om, float *k, float *nu, float *ir) {
        *om = p.omega_f;
        *k = p.k_f;
        *nu = p.nu_f;
        *ir = __ldg(&p.inv_r_f[j]);
    }
};
template <> struct Consts<double> {
    static __device__ __forceinline__ void get(const Params &p, int j, double *om, double *k, double *nu, double *ir) {
        *om = p.omega_d;
        *k = p.k_d;
        *nu = p.nu_d;
        *ir = __ldg(&p.inv_r_d[j]);
    }
};

struct BcDev {
    int n_bc;
    const BcParam *par;     // kind, sign, par[], period, etab_off, q_scale used
    BcState *state;
    const double *etab;
    const double *profile;  // 3 per boundary node
    const int32_t *xf_off, *xf_n, *xf;      // first-layer nodes per boundary
    const double *area;                     // 2 pi r per first-layer node (in xf order)
    const double *area_sum;                 // per boundary
    const int32_t *lk_off, *lk_n;           // links per boundary
    const int32_t *lk_xf, *lk_ieff, *lk_xb, *lk_ib, *lk_node, *lk_xfi;
    const int32_t *node_off;                // first profile row per boundary
    double *v0;                             // 2 per first-layer node
    double *wave;                           // ring [cap][1 + 4 n_bc]
    int wave_cap;
    long long *step;                        // index t_n of the step in progress
    // the boundary work of a step as two kernels: k_axi_bc_reduce (block k sums
    // the first-layer chunk red_chunk[k] of boundary red_bc[k] into a partial)
    // and k_axi_bc_apply (block k takes the 0D step of boundary app_bc[k] from
    // the partials, summed in a fixed order, and writes the ghosts of its link
    // chunk app_chunk[k]); state is [2][n_bc]: step t reads slot t & 1 and
    // writes slot (t + 1) & 1
    double *partial;                        // 2 per reduce block
    const int32_t *red_bc, *red_chunk, *red_off, *red_n, *app_bc, *app_chunk;
    int n_red_blocks, n_app_blocks;
};

// grid: (x-blocks, nr) of 256 nodes of a row, one row of the (x, r) grid per
// blockIdx.y; the launch covers the x-blocks xb0 .. xb0 + gridDim.x - 1
template <class S>
__global__ void __launch_bounds__(256, 8) k_axi_collide(const S *__restrict__ fin, S *__restrict__ fout, Params p,
                                                       int xb0) {
    using R = typename Storage<S>::R;
    const int x = (blockIdx.x + xb0) * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (p.step && x == 0 && j == 0) *p.step += 1;  // the step index t_n seen by the boundary kernels
    if (x >= p.nx) return;
    const int c = j * p.nx + x;
    const uint32_t fl = __ldg(&p.flags[c]);
    if (!(fl & AF_FLUID)) return;
    const int n = p.n;
    R s[Q9];
#pragma unroll
    for (int i = 0; i < Q9; i++) {
        uint32_t src;
        if (i == 0) src = (uint32_t)c;
        else if (fl & (1u << i)) src = (uint32_t)(opp(i) * n + c);
        else if (j - er(i) < 0) src = (uint32_t)(mir(i) * n + (x - ex(i)));  // mirror at the axis (row 0)
        else src = (uint32_t)(i * n + c - ex(i) - er(i) * p.nx);
        s[i] = Storage<S>::ld(fin + src);
    }
    // moments from the sums and differences of the four opposite pairs
    // (1, 2) = +-e_x, (3, 4) = +-e_r, (5, 6) = +-(e_x + e_r), (7, 8) = +-(e_x - e_r)
    R Sp[4], Dp[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        Sp[q] = s[2 * q + 1] + s[2 * q + 2];
        Dp[q] = s[2 * q + 1] - s[2 * q + 2];
    }
    const R sd = s[0] + ((Sp[0] + Sp[1]) + (Sp[2] + Sp[3]));
    const R jx = Dp[0] + Dp[2] + Dp[3], jr = Dp[1] + Dp[2] - Dp[3];
    const R pxr = Sp[2] - Sp[3], prr = Sp[1] + Sp[2] + Sp[3];
    R omega, k, nu, inv_r;
    Consts<R>::get(p, j, &omega, &k, &nu, &inv_r);
    const R m = -jr * inv_r;
    const R sp = sd + R(0.5) * m;                       // 3P - 1
    // non-equilibrium stress of f against f^eq(c_s^2 sum f, j): Pi^eq_xr = j_x j_r,
    // Pi^eq_rr = c_s^2 sum f + j_r^2 (sum f = 1 + sd)
    const R Pi_xr = pxr - jx * jr;
    const R Pi_rr = prr - sd / R(3) - jr * jr;
    const R gx = -k * Pi_xr * inv_r - jx * jr * inv_r;
    const R gr = -k * Pi_rr * inv_r - R(2) * nu * jr * inv_r * inv_r - jr * jr * inv_r;
    const R vx = jx + R(0.5) * gx, vr = jr + R(0.5) * gr;
    const R vv = vx * vx + vr * vr;
    if (!(sd - sd == R(0)) || !(vv <= R(0.09))) atomicOr(p.status, 1u);
    if (fl & AF_XF) {
        R *aux = static_cast<R *>(p.aux);
        aux[c] = sp;
        aux[n + c] = jx;
        aux[2 * n + c] = jr;
        aux[3 * n + c] = vx;
        aux[4 * n + c] = vr;
        aux[5 * n + c] = sd;
    }
    // BGK with f^eq_i - w_i = w_i (sp + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2), the Guo
    // term k w_i (3 (e - v).g + 9 (e.v)(e.g)) and the mass source k w_i m,
    // k = 1 - 1/(2 tau), written per opposite pair (e.v and e.g change sign):
    //   s*_i = (1 - omega) s_i + w (A + B),  s*_i' = (1 - omega) s_i' + w (A - B),
    //   A = A0 + e.v (9/2 omega e.v + 9 k e.g),  B = 3 omega e.v + 3 k e.g,
    //   A0 = omega (sp - 3/2 v^2) + k (m - 3 v.g)
    const R om1 = R(1) - omega;
    const R A0 = omega * (sp - R(1.5) * vv) + k * (m - R(3) * (vx * gx + vr * gr));
    const R c45 = R(4.5) * omega, c9 = R(9) * k, c3w = R(3) * omega, c3k = R(3) * k;
    const R eu[4] = {vx, vr, vx + vr, vx - vr};
    const R eg[4] = {gx, gr, gx + gr, gx - gr};
    Storage<S>::st(fout + (uint32_t)c, om1 * s[0] + R(4.0 / 9.0) * A0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const R w = q < 2 ? R(1.0 / 9.0) : R(1.0 / 36.0);
        const R A = A0 + eu[q] * (c45 * eu[q] + c9 * eg[q]);
        const R B = c3w * eu[q] + c3k * eg[q];
        const int i = 2 * q + 1;
        Storage<S>::st(fout + ((uint32_t)i * (uint32_t)n + (uint32_t)c), om1 * s[i] + w * (A + B));  // 9 n < 2^31
        Storage<S>::st(fout + ((uint32_t)(i + 1) * (uint32_t)n + (uint32_t)c), om1 * s[i + 1] + w * (A - B));
    }
}

// f(t_n) (pulled) and P, u_x, u_r at every node; zero off the fluid
template <class S>
__global__ void k_axi_gather(const S *__restrict__ fin, Params p, double *f9, double *mac3) {
    using R = typename Storage<S>::R;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n) return;
    const uint32_t fl = p.flags[c];
    const int n = p.n, x = c % p.nx, j = c / p.nx;
    if (!(fl & AF_FLUID)) {
        for (int i = 0; i < Q9; i++) f9[(size_t)i * n + c] = 0.0;
        mac3[c] = mac3[n + c] = mac3[2 * n + c] = 0.0;
        return;
    }
    double s[Q9], sd = 0, jx = 0, jr = 0, pxr = 0, prr = 0;
    for (int i = 0; i < Q9; i++) {
        int src;
        if (i == 0) src = c;
        else if (fl & (1u << i)) src = opp(i) * n + c;
        else if (j - er(i) < 0) src = mir(i) * n + (x - ex(i));
        else src = i * n + c - ex(i) - er(i) * p.nx;
        s[i] = (double)Storage<S>::ld(fin + src);
        f9[(size_t)i * n + c] = s[i] + wgt(i);
        sd += s[i];
        jx += ex(i) * s[i];
        jr += er(i) * s[i];
        prr += er(i) * er(i) * s[i];
        pxr += ex(i) * er(i) * s[i];
    }
    const double tau = p.tau, k = 1.0 - 0.5 / tau, nu = (tau - 0.5) / 3.0, inv_r = 1.0 / (j + 0.5);
    const double m = -jr * inv_r, sp = sd + 0.5 * m;
    const double gx = -k * (pxr - jx * jr) * inv_r - jx * jr * inv_r;
    const double gr = -k * (prr - sd / 3.0 - jr * jr) * inv_r - 2.0 * nu * jr * inv_r * inv_r - jr * jr * inv_r;
    mac3[c] = (1.0 + sp) / 3.0;
    mac3[n + c] = jx + 0.5 * gx;
    mac3[2 * n + c] = jr + 0.5 * gr;
}

// lays out f(t_0) so that the next pull reads it: the population i of node c
// is stored where the pull of (c, i) looks for it
template <class S>
__global__ void k_axi_init(S *__restrict__ fout, Params p, const double *__restrict__ f9) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n) return;
    const uint32_t fl = p.flags[c];
    if (!(fl & AF_FLUID)) return;
    const int n = p.n, x = c % p.nx, j = c / p.nx;
    for (int i = 0; i < Q9; i++) {
        int src;
        if (i == 0) src = c;
        else if (fl & (1u << i)) src = opp(i) * n + c;
        else if (j - er(i) < 0) src = mir(i) * n + (x - ex(i));
        else src = i * n + c - ex(i) - er(i) * p.nx;
        Storage<S>::st(fout + src, (typename Storage<S>::R)(f9[(size_t)i * n + c] - wgt(i)));
    }
}

// f^eq_i(P*, v*) - f^eq_i(P, v) with 3P - 1 = sp (in the compute type R)
template <class R>
__device__ __forceinline__ R dfeq_dev(int i, R sps, R vxs, R vrs, R spf, R vxf, R vrf) {
    const R eus = R(ex(i)) * vxs + R(er(i)) * vrs, euf = R(ex(i)) * vxf + R(er(i)) * vrf;
    const R w = (R)wgt(i);
    return w * (sps - spf) +
           w * (R(3) * (eus - euf) + R(4.5) * (eus * eus - euf * euf) -
                R(1.5) * ((vxs * vxs + vrs * vrs) - (vxf * vxf + vrf * vrf)));
}

// The 0D boundaries in two kernels.  k_axi_bc_reduce: block k sums, over
// its chunk of BC2 first-layer nodes of boundary red_bc[k], the area-weighted
// flow n.j / sum f and pressure deviation in FP64 (per-node terms in the
// compute type), tree-reduced in shared memory, into partial[k].
// k_axi_bc_apply: block k sums the partials of boundary app_bc[k] in their
// fixed order on one thread, takes the 0D step (t_n -> t_{n+1}) there (every
// link block of the boundary takes the same step from the same state slot,
// same bits; its first block stores the new state and the waveform row), and
// writes the ghosts of its chunk of links, Eq. Non-equilibrium3 written as
//   f_i(x_b) = f*_i'(x_f) + f^eq_i'(P*, v*) - f^eq_i'(P(x_f), v(x_f)),
// i' the direction arriving at x_f (mirrored for links across the axis).  A
// valve closing in this step prescribes v_0(T_d) = v(x_f, T_d) per link
// (links sharing x_f store the same closure velocity).  Pressures are
// deviations from P_ref (the FP64 pipe of this part is narrow); the sums and
// the 0D step are FP64.
constexpr int BC2 = 256;

template <class S>
__global__ void __launch_bounds__(BC2) k_axi_bc_reduce(Params p, BcDev q) {
    using R = typename Storage<S>::R;
    const R *aux = static_cast<const R *>(p.aux);
    const int n = p.n;
    const int b = q.red_bc[blockIdx.x], ch = q.red_chunk[blockIdx.x];
    const BcParam &P = q.par[b];
    __shared__ double sQ[BC2], sP[BC2];
    double Q = 0.0, Ps = 0.0;  // Ps: sum of A (P - P_ref)
    const int a = ch * BC2 + threadIdx.x;
    if (a < q.xf_n[b]) {
        const int cf = q.xf[q.xf_off[b] + a];
        const R A = (R)q.area[q.xf_off[b] + a];
        Q = (double)(A * (R)P.sign * aux[n + cf] / (R(1) + aux[5 * n + cf]));
        Ps = (double)(A * aux[cf] / R(3));
    }
    sQ[threadIdx.x] = Q;
    sP[threadIdx.x] = Ps;
    __syncthreads();
    for (int st = BC2 / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            sQ[threadIdx.x] += sQ[threadIdx.x + st];
            sP[threadIdx.x] += sP[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        q.partial[2 * blockIdx.x] = sQ[0];
        q.partial[2 * blockIdx.x + 1] = sP[0];
    }
}

template <class S>
__global__ void __launch_bounds__(BC2) k_axi_bc_apply(S *__restrict__ f, Params p, BcDev q) {
    using R = typename Storage<S>::R;
    const R *aux = static_cast<const R *>(p.aux);
    const int n = p.n;
    const int b = q.app_bc[blockIdx.x], ch = q.app_chunk[blockIdx.x];
    const BcParam &P = q.par[b];
    const long long t = *q.step;
    __shared__ double sh_Pstar, sh_S, sh_cos, sh_sin;
    __shared__ int sh_ptype, sh_closed;
    if (threadIdx.x == 0) {
        double Q = 0.0, Ps = 0.0;
        for (int k = 0; k < q.red_n[b]; k++) {  // the partials in their fixed order
            Q += q.partial[2 * (q.red_off[b] + k)];
            Ps += q.partial[2 * (q.red_off[b] + k) + 1];
        }
        int ptype, closed;
        double Sm;
        const double Psum = q.area_sum[b] / 3.0 + Ps;  // sum of A P over the layer
        const BcState st = zero_d_step(P, q.state[(size_t)(t & 1) * q.n_bc + b], Q, Psum, q.area_sum[b], t, q.etab,
                                       &ptype, &closed, &Sm);
        sh_Pstar = st.Pstar_gauge;
        sh_ptype = ptype;
        sh_closed = closed;
        sh_S = Sm;
        if (P.kind == BC_VELOCITY) {  // the inlet's phase, once per block
            const double w = P.par[0], tn1 = (double)(t + 1);
            sh_cos = cos(w * tn1);
            sh_sin = sin(w * tn1);
        }
        if (ch == 0) {
            q.state[(size_t)((t + 1) & 1) * q.n_bc + b] = st;
            const int width = 1 + 4 * q.n_bc;
            double *row = q.wave + (size_t)(t % q.wave_cap) * width;
            if (b == 0) row[0] = (double)t;
            row[1 + 4 * b] = st.Qu;
            row[2 + 4 * b] = st.Pbar - 1.0 / 3.0;
            row[3 + 4 * b] = P.kind == BC_RCR ? st.Pw : (P.kind == BC_LV ? st.Pv : st.Pstar_gauge);
            row[4 + 4 * b] = st.valve_open;
        }
    }
    __syncthreads();
    const int L = ch * BC2 + threadIdx.x;
    if (L >= q.lk_n[b]) return;
    const int g = q.lk_off[b] + L;
    const int cf = q.lk_xf[g], ie = q.lk_ieff[g];
    const R spf = aux[cf], vxf = aux[3 * n + cf], vrf = aux[4 * n + cf];
    R sps, vxs, vrs;
    if (sh_ptype) {
        sps = (R)(3.0 * sh_Pstar);  // 3 P* - 1 with P* = P_ref + P*_gauge
        vxs = vxf;
        vrs = vrf;
    } else if (P.kind == BC_VELOCITY) {
        const double *pr = q.profile + 3 * (size_t)(q.node_off[b] + q.lk_node[g]);
        sps = spf;
        vxs = (R)((double)P.sign * (pr[0] + pr[1] * sh_cos - pr[2] * sh_sin));
        vrs = R(0);
    } else {
        double *v0 = q.v0 + 2 * (size_t)(q.xf_off[b] + q.lk_xfi[g]);
        double u0x, u0r;
        if (sh_closed) {  // v_0(T_d) = v(x_f, T_d)
            u0x = (double)vxf;
            u0r = (double)vrf;
            v0[0] = u0x;
            v0[1] = u0r;
        } else {
            u0x = v0[0];
            u0r = v0[1];
        }
        sps = spf;
        vxs = (R)(u0x * sh_S);
        vrs = (R)(u0r * sh_S);
    }
    const R ghost = Storage<S>::ld(f + (size_t)ie * n + cf) + dfeq_dev<R>(ie, sps, vxs, vrs, spf, vxf, vrf);
    Storage<S>::st(f + (size_t)q.lk_ib[g] * n + q.lk_xb[g], ghost);
}

}  // namespace axi
}  // namespace lbm

using namespace lbm;
using namespace lbm::axi;

struct lbm_axi_handle {
    int device = 0, prec = 0, nx = 0, nr = 0, n = 0;
    double tau = 0.8;
    int q_scale = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int graph_steps = 64, wave_cap = 8192;
    cudaGraphExec_t graph = nullptr;
    // Inside the step graph, the collide of the next step over the x-blocks
    // that hold no first-layer node, [xb_lo, xb_hi) (they pull no ghost and
    // write no aux), runs beside this step's boundary kernels (stream s_bc);
    // the edge x-blocks follow the boundary kernels.  xb_hi = 0: no split.
    int xb_lo = 0, xb_hi = 0;
    cudaStream_t s_bc = nullptr;
    cudaEvent_t ev_f = nullptr, ev_d = nullptr;
    int parity = 0;
    int64_t steps = 0;
    void *f[2] = {nullptr, nullptr};
    uint16_t *flags = nullptr;
    void *aux = nullptr;
    unsigned *status = nullptr;
    long long *d_step = nullptr;
    double *rd = nullptr;  // read-out scratch (12 n doubles)
    float *inv_r_f = nullptr;
    double *inv_r_d = nullptr;
    // boundaries (host copies kept for read-out)
    std::vector<BcParam> bcp;
    std::vector<double> etab_h;
    BcDev bd{};
    std::vector<void *> allocs;
    std::string err;
};

namespace {

lbm_status afail(lbm_axi_handle *h, lbm_status s, const std::string &m) {
    if (h) h->err = m;
    return s;
}

#define ACK(h, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return afail(h, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T> cudaError_t aalloc(lbm_axi_handle *h, T **p, size_t count) {
    *p = nullptr;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

template <class T> cudaError_t aupload(lbm_axi_handle *h, T **p, const std::vector<T> &v) {
    cudaError_t e = aalloc(h, p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

Params params(const lbm_axi_handle *h) {
    Params p;
    p.nx = h->nx;
    p.nr = h->nr;
    p.n = h->n;
    p.flags = h->flags;
    p.aux = h->aux;
    p.tau = h->tau;
    p.status = h->status;
    p.omega_d = 1.0 / h->tau;
    p.k_d = 1.0 - 0.5 / h->tau;
    p.nu_d = (h->tau - 0.5) / 3.0;
    p.omega_f = (float)p.omega_d;
    p.k_f = (float)p.k_d;
    p.nu_f = (float)p.nu_d;
    p.inv_r_f = h->inv_r_f;
    p.inv_r_d = h->inv_r_d;
    p.step = h->d_step;
    return p;
}

template <class S> cudaError_t collide_blocks(lbm_axi_handle *h, const void *fin, void *fout, int b0, int b1,
                                              cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    k_axi_collide<S><<<dim3(b1 - b0, h->nr), 256, 0, st>>>(static_cast<const S *>(fin), static_cast<S *>(fout),
                                                         params(h), b0);
    return cudaGetLastError();
}

template <class S> cudaError_t bc_kernels(lbm_axi_handle *h, void *fout, cudaStream_t st) {
    if (!h->bd.n_bc) return cudaSuccess;
    const Params p = params(h);
    k_axi_bc_reduce<S><<<h->bd.n_red_blocks, BC2, 0, st>>>(p, h->bd);
    k_axi_bc_apply<S><<<h->bd.n_app_blocks, BC2, 0, st>>>(static_cast<S *>(fout), p, h->bd);
    return cudaGetLastError();
}

// One step.  pre: the interior x-blocks of this step's collide were issued by
// the previous step; next: issue the next step's interior x-blocks beside
// this step's boundary kernels (graph capture only).
template <class S> cudaError_t launch_step_t(lbm_axi_handle *h, bool pre, bool next) {
    const int nbx = (h->nx + 255) / 256;
    void *fin = h->f[h->parity], *fout = h->f[1 - h->parity];
    cudaError_t e = cudaSuccess;
    if (pre) {  // the edge x-blocks, once the previous step's ghosts are in place
        e = cudaStreamWaitEvent(h->stream, h->ev_d, 0);
        if (e == cudaSuccess) e = collide_blocks<S>(h, fin, fout, 0, h->xb_lo, h->stream);
        if (e == cudaSuccess) e = collide_blocks<S>(h, fin, fout, h->xb_hi, nbx, h->stream);
    } else {
        e = collide_blocks<S>(h, fin, fout, 0, nbx, h->stream);
    }
    if (e != cudaSuccess) return e;
    if (next) {
        e = cudaEventRecord(h->ev_f, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_bc, h->ev_f, 0);
        if (e == cudaSuccess) e = bc_kernels<S>(h, fout, h->s_bc);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_d, h->s_bc);
        // the next step reads fout and writes fin
        if (e == cudaSuccess) e = collide_blocks<S>(h, fout, fin, h->xb_lo, h->xb_hi, h->stream);
    } else {
        e = bc_kernels<S>(h, fout, h->stream);
    }
    h->parity = 1 - h->parity;
    return e;
}

cudaError_t launch_step(lbm_axi_handle *h, bool pre = false, bool next = false) {
    return h->prec == LBM_F64 ? launch_step_t<double>(h, pre, next) : launch_step_t<float>(h, pre, next);
}

// step counter for graph-free steps (the boundary kernel advances it when
// there are boundaries; without boundaries nothing reads it)
void count_step(lbm_axi_handle *h) { h->steps++; }

}  // namespace

extern "C" {

lbm_status lbm_axi_create(const lbm_axi_config *cfg, lbm_axi_handle **out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!cfg || !cfg->node || cfg->nx < 3 || cfg->nr < 1 || !(cfg->tau > 0.5) || cfg->n_bc < 0 || cfg->n_bc > 8 ||
        (cfg->n_bc > 0 && !cfg->bc) || (cfg->precision != LBM_F32 && cfg->precision != LBM_F64) ||
        cfg->graph_steps < 0 || (cfg->graph_steps % 2) != 0 || (int64_t)cfg->nx * cfg->nr * 9 >= 2147483647LL) {
        fprintf(stderr, "lbm_axi_create: invalid configuration\n");
        return LBM_ERR_ARG;
    }
    const int nx = cfg->nx, nr = cfg->nr, n = nx * nr;
    const uint8_t *node = cfg->node;
    // validate boundaries
    for (int k = 0; k < cfg->n_bc; k++) {
        const lbm_boundary_desc &b = cfg->bc[k];
        if (b.axis != 0 || (b.sign != 1 && b.sign != -1) || b.kind < 0 || b.kind > 3 || b.n_params < 1 || !b.params) {
            fprintf(stderr, "lbm_axi_create: boundary %d: axis must be 0, sign +-1, params given\n", k);
            return LBM_ERR_ARG;
        }
        const int col = b.sign > 0 ? 0 : nx - 1;
        int cnt = 0;
        for (int j = 0; j < nr; j++)
            for (int x = 0; x < nx; x++)
                if (node[j * nx + x] == 2 + k) {
                    if (x != col) {
                        fprintf(stderr, "lbm_axi_create: boundary %d node off its column\n", k);
                        return LBM_ERR_ARG;
                    }
                    cnt++;
                }
        if ((b.kind == LBM_BC_RCR || b.kind == LBM_BC_LV) && b.n_params < 4) return LBM_ERR_ARG;
        if (b.kind == LBM_BC_VELOCITY && (!b.profile || b.n_profile != cnt)) return LBM_ERR_ARG;
        if (b.kind == LBM_BC_LV && (b.period <= 0 || !b.elastance || (int)b.params[0] != b.period || !(b.params[2] > 0)))
            return LBM_ERR_ARG;
        if (b.n_params > 4 && !(b.params[4] == 1 || b.params[4] == 2 || b.params[4] == 4)) return LBM_ERR_ARG;
    }
    for (int c = 0; c < n; c++)
        if (node[c] > 1 && node[c] - 2 >= cfg->n_bc) {
            fprintf(stderr, "lbm_axi_create: node code without a boundary\n");
            return LBM_ERR_ARG;
        }
    lbm_axi_handle *h = new lbm_axi_handle();
    h->device = cfg->device;
    h->prec = cfg->precision;
    h->nx = nx;
    h->nr = nr;
    h->n = n;
    h->tau = cfg->tau;
    h->q_scale = cfg->q_scale;
    h->graph_steps = cfg->graph_steps ? cfg->graph_steps : 64;
    h->wave_cap = cfg->wave_capacity > 0 ? cfg->wave_capacity : 8192;
    auto bail = [&](const std::string &m) {
        fprintf(stderr, "lbm_axi_create: %s\n", m.c_str());
        lbm_axi_destroy(h);
        return LBM_ERR_CUDA;
    };
    // flags and pull sources on the host
    auto is_wall = [&](int x, int j) { return x < 0 || x >= nx || j >= nr || node[j * nx + x] == 1; };
    std::vector<uint16_t> flags(n, 0);
    for (int j = 0; j < nr; j++)
        for (int x = 0; x < nx; x++) {
            const int c = j * nx + x;
            if (node[c] != 0) continue;
            uint16_t fl = AF_FLUID;
            for (int i = 1; i < Q9; i++) {
                int xs = x - ex(i), js = j - er(i);
                if (js < 0) js = 0;  // mirror image row
                if (is_wall(xs, js)) fl |= (uint16_t)(1u << i);
            }
            flags[c] = fl;
        }
    // boundaries: nodes, links, first layer
    std::vector<BcParam> bcp;
    std::vector<int32_t> xf_off, xf_n, xf, lk_off, lk_n, lk_xf, lk_ieff, lk_xb, lk_ib, lk_node, lk_xfi, node_off;
    std::vector<double> area, area_sum, profile, etab;
    for (int k = 0; k < cfg->n_bc; k++) {
        const lbm_boundary_desc &b = cfg->bc[k];
        const int code = 2 + k;
        std::vector<int> nodes_of(n, -1);
        int cnt = 0;
        for (int j = 0; j < nr; j++)
            for (int x = 0; x < nx; x++)
                if (node[j * nx + x] == code) nodes_of[j * nx + x] = cnt++;
        node_off.push_back((int32_t)(profile.size() / 3));
        if (b.kind == LBM_BC_VELOCITY)
            for (int a = 0; a < 3 * cnt; a++) profile.push_back(b.profile[a]);
        struct Lk { int xf, ie, xb, ib, nd; };
        std::vector<Lk> lks;
        for (int j = 0; j < nr; j++)
            for (int x = 0; x < nx; x++) {
                const int c = j * nx + x;
                if (node[c] != 0) continue;
                for (int i = 1; i < Q9; i++) {
                    if (flags[c] & (1u << i)) continue;
                    int xs = x - ex(i), js = j - er(i), ii = i;
                    if (js < 0) {
                        js = 0;
                        ii = mir(i);
                    }
                    const int cs = js * nx + xs;
                    if (node[cs] == code) lks.push_back({c, i, cs, ii, nodes_of[cs]});
                }
            }
        // first layer in (j, x) order
        std::vector<int> cells;
        for (auto &l : lks) cells.push_back(l.xf);
        std::sort(cells.begin(), cells.end());
        cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
        xf_off.push_back((int32_t)xf.size());
        xf_n.push_back((int32_t)cells.size());
        double A = 0.0;
        for (int cf : cells) {
            xf.push_back(cf);
            const double a = 2.0 * 3.14159265358979323846 * ((cf / nx) + 0.5);
            area.push_back(a);
            A += a;
        }
        area_sum.push_back(A);
        lk_off.push_back((int32_t)lk_xf.size());
        lk_n.push_back((int32_t)lks.size());
        for (auto &l : lks) {
            lk_xf.push_back(l.xf);
            lk_ieff.push_back(l.ie);
            lk_xb.push_back(l.xb);
            lk_ib.push_back(l.ib);
            lk_node.push_back(l.nd);
            lk_xfi.push_back((int32_t)(std::lower_bound(cells.begin(), cells.end(), l.xf) - cells.begin()));
        }
        BcParam P;
        memset(&P, 0, sizeof P);
        P.kind = b.kind;
        P.axis = 0;
        P.sign = b.sign;
        P.n_xf = (int)cells.size();
        P.q_scale = cfg->q_scale;
        for (int a = 0; a < std::min(b.n_params, 8); a++) P.par[a] = b.params[a];
        if (b.kind == LBM_BC_LV) {
            P.period = b.period;
            P.etab_off = (int)(etab.size() / 2);
            for (int a = 0; a < 2 * b.period; a++) etab.push_back(b.elastance[a]);
        }
        bcp.push_back(P);
    }
    for (int32_t cf : xf) flags[cf] |= AF_XF;
    std::vector<BcState> st(bcp.size());
    for (size_t k = 0; k < bcp.size(); k++) {
        memset(&st[k], 0, sizeof(BcState));
        st[k].Pbar = 1.0 / 3.0;
        if (bcp[k].kind == BC_RCR) st[k].Pw = bcp[k].par[3];
        if (bcp[k].kind == BC_LV) {
            st[k].Pv = bcp[k].par[3];
            st[k].Td = -1e300;
        }
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return bail("cudaSetDevice failed");
    if (cfg->stream) h->stream = static_cast<cudaStream_t>(cfg->stream);
    else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail("stream");
        h->own_stream = true;
    }
    const size_t sb = h->prec == LBM_F64 ? 8 : 4;
    for (int k = 0; k < 2; k++) {
        uint8_t *q;
        if (aalloc(h, &q, (size_t)Q9 * n * sb) != cudaSuccess || cudaMemset(q, 0, (size_t)Q9 * n * sb) != cudaSuccess)
            return bail("out of memory (populations)");
        h->f[k] = q;
    }
    uint8_t *aq;
    if (aupload(h, &h->flags, flags) != cudaSuccess || aalloc(h, &aq, (size_t)6 * n * sb) != cudaSuccess ||
        cudaMemset(aq, 0, (size_t)6 * n * sb) != cudaSuccess || aalloc(h, &h->status, 1) != cudaSuccess ||
        cudaMemset(h->status, 0, sizeof(unsigned)) != cudaSuccess || aalloc(h, &h->d_step, 1) != cudaSuccess ||
        cudaMemset(h->d_step, 0xff, sizeof(long long)) != cudaSuccess ||  // -1: the first collide makes it t_0 = 0
        aalloc(h, &h->rd, (size_t)12 * n) != cudaSuccess)
        return bail("out of memory");
    h->aux = aq;
    {
        std::vector<double> ird(nr);
        std::vector<float> irf(nr);
        for (int j = 0; j < nr; j++) {
            ird[j] = 1.0 / (j + 0.5);
            irf[j] = (float)(1.0 / (j + 0.5));
        }
        if (aupload(h, &h->inv_r_d, ird) != cudaSuccess || aupload(h, &h->inv_r_f, irf) != cudaSuccess)
            return bail("out of memory");
    }
    h->bcp = bcp;
    h->etab_h = etab;
    BcDev &bd = h->bd;
    bd.n_bc = (int)bcp.size();
    BcParam *dpar;
    BcState *dst;
    double *dv0, *dwave;
    const size_t width = 1 + 4 * std::max<size_t>(bcp.size(), 1);
    std::vector<BcState> st2(st);  // both slots of the state start equal
    st2.insert(st2.end(), st.begin(), st.end());
    std::vector<int32_t> red_bc, red_chunk, red_off, red_n, app_bc, app_chunk;
    for (size_t b = 0; b < bcp.size(); b++) {
        const int nr = std::max(1, (xf_n[b] + BC2 - 1) / BC2), na = std::max(1, (lk_n[b] + BC2 - 1) / BC2);
        red_off.push_back((int32_t)red_bc.size());
        red_n.push_back(nr);
        for (int k = 0; k < nr; k++) {
            red_bc.push_back((int32_t)b);
            red_chunk.push_back(k);
        }
        for (int k = 0; k < na; k++) {
            app_bc.push_back((int32_t)b);
            app_chunk.push_back(k);
        }
    }
    double *dpart = nullptr;
    bool ok = aupload(h, &dpar, bcp) == cudaSuccess && aupload(h, &dst, st2) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.red_bc, red_bc) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.red_chunk, red_chunk) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.red_off, red_off) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.red_n, red_n) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.app_bc, app_bc) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.app_chunk, app_chunk) == cudaSuccess &&
              aalloc(h, &dpart, 2 * std::max<size_t>(red_bc.size(), 1)) == cudaSuccess &&
              aupload(h, (double **)&bd.etab, etab) == cudaSuccess &&
              aupload(h, (double **)&bd.profile, profile) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.xf_off, xf_off) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.xf_n, xf_n) == cudaSuccess && aupload(h, (int32_t **)&bd.xf, xf) == cudaSuccess &&
              aupload(h, (double **)&bd.area, area) == cudaSuccess &&
              aupload(h, (double **)&bd.area_sum, area_sum) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_off, lk_off) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_n, lk_n) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_xf, lk_xf) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_ieff, lk_ieff) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_xb, lk_xb) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_ib, lk_ib) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_node, lk_node) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.lk_xfi, lk_xfi) == cudaSuccess &&
              aupload(h, (int32_t **)&bd.node_off, node_off) == cudaSuccess &&
              aalloc(h, &dv0, 2 * std::max<size_t>(xf.size(), 1)) == cudaSuccess &&
              cudaMemset(dv0, 0, 2 * std::max<size_t>(xf.size(), 1) * sizeof(double)) == cudaSuccess &&
              aalloc(h, &dwave, (size_t)h->wave_cap * width) == cudaSuccess &&
              cudaMemset(dwave, 0, (size_t)h->wave_cap * width * sizeof(double)) == cudaSuccess;
    if (!ok) return bail("out of memory (boundaries)");
    bd.par = dpar;
    bd.state = dst;
    bd.partial = dpart;
    bd.n_red_blocks = (int)red_bc.size();
    bd.n_app_blocks = (int)app_bc.size();
    bd.v0 = dv0;
    bd.wave = dwave;
    bd.wave_cap = h->wave_cap;
    bd.step = h->d_step;
    if (!bcp.empty()) {
        // x-blocks holding a first-layer node (the only nodes that pull ghosts
        // or write aux) must wait for the boundary kernels; the rest may not
        const int nbx = (nx + 255) / 256;
        std::vector<uint8_t> edge((size_t)nbx, 0);
        for (int32_t c : xf) edge[(size_t)((c % nx) / 256)] = 1;
        int lo = 0, hi = nbx;
        while (lo < nbx && edge[(size_t)lo]) lo++;
        while (hi > lo && edge[(size_t)(hi - 1)]) hi--;
        bool inner_clear = hi > lo;
        for (int b = lo; b < hi; b++) inner_clear = inner_clear && !edge[(size_t)b];
        if (inner_clear) {
            int plo = 0, phi = 0;
            if (cudaDeviceGetStreamPriorityRange(&plo, &phi) != cudaSuccess ||
                cudaStreamCreateWithPriority(&h->s_bc, cudaStreamNonBlocking, phi) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_f, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_d, cudaEventDisableTiming) != cudaSuccess)
                return bail("streams");
            h->xb_lo = lo;
            h->xb_hi = hi;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return bail("initialisation failed");
    *out = h;
    return LBM_OK;
}

lbm_status lbm_axi_step(lbm_axi_handle *h, int64_t nsteps) {
    if (!h || nsteps < 0) return afail(h, LBM_ERR_ARG, "bad arguments");
    ACK(h, cudaSetDevice(h->device));
    int64_t done = 0;
    while (done < nsteps) {
        const int64_t left = nsteps - done;
        if (h->parity == 0 && left >= h->graph_steps) {
            if (!h->graph) {
                cudaGraph_t g;
                ACK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
                const bool split = h->xb_hi > h->xb_lo;
                for (int k = 0; k < h->graph_steps; k++) {
                    cudaError_t e = launch_step(h, split && k > 0, split && k + 1 < h->graph_steps);
                    if (e != cudaSuccess) {
                        cudaStreamEndCapture(h->stream, &g);
                        return afail(h, LBM_ERR_CUDA, cudaGetErrorString(e));
                    }
                }
                ACK(h, cudaStreamEndCapture(h->stream, &g));
                ACK(h, cudaGraphInstantiate(&h->graph, g, 0));
                cudaGraphDestroy(g);
            }
            ACK(h, cudaGraphLaunch(h->graph, h->stream));
            done += h->graph_steps;
            h->steps += h->graph_steps;
        } else {
            ACK(h, launch_step(h));
            done++;
            count_step(h);
        }
    }
    return LBM_OK;
}

lbm_status lbm_axi_sync(lbm_axi_handle *h) {
    if (!h) return LBM_ERR_ARG;
    ACK(h, cudaSetDevice(h->device));
    ACK(h, cudaStreamSynchronize(h->stream));
    unsigned st = 0;
    ACK(h, cudaMemcpy(&st, h->status, sizeof st, cudaMemcpyDeviceToHost));
    if (st) return afail(h, LBM_ERR_UNSTABLE, "NaN/Inf or |v| > 0.3 in the lattice");
    return LBM_OK;
}

static lbm_status gather(lbm_axi_handle *h) {
    ACK(h, cudaSetDevice(h->device));
    const Params p = params(h);
    const int grid = (h->n + 255) / 256;
    if (h->prec == LBM_F64)
        k_axi_gather<double><<<grid, 256, 0, h->stream>>>(static_cast<const double *>(h->f[h->parity]), p, h->rd,
                                                          h->rd + (size_t)Q9 * h->n);
    else
        k_axi_gather<float><<<grid, 256, 0, h->stream>>>(static_cast<const float *>(h->f[h->parity]), p, h->rd,
                                                         h->rd + (size_t)Q9 * h->n);
    ACK(h, cudaGetLastError());
    ACK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_axi_read_fields(lbm_axi_handle *h, double *P, double *ux, double *ur) {
    if (!h || !P || !ux || !ur) return afail(h, LBM_ERR_ARG, "null array");
    lbm_status s = gather(h);
    if (s != LBM_OK) return s;
    const size_t n = h->n, o = (size_t)Q9 * n;
    ACK(h, cudaMemcpy(P, h->rd + o, n * sizeof(double), cudaMemcpyDeviceToHost));
    ACK(h, cudaMemcpy(ux, h->rd + o + n, n * sizeof(double), cudaMemcpyDeviceToHost));
    ACK(h, cudaMemcpy(ur, h->rd + o + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_axi_read_populations(lbm_axi_handle *h, double *f) {
    if (!h || !f) return afail(h, LBM_ERR_ARG, "null array");
    lbm_status s = gather(h);
    if (s != LBM_OK) return s;
    ACK(h, cudaMemcpy(f, h->rd, (size_t)Q9 * h->n * sizeof(double), cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_axi_init_populations(lbm_axi_handle *h, const double *f) {
    if (!h || !f) return afail(h, LBM_ERR_ARG, "null array");
    ACK(h, cudaSetDevice(h->device));
    ACK(h, cudaStreamSynchronize(h->stream));
    ACK(h, cudaMemcpy(h->rd, f, (size_t)Q9 * h->n * sizeof(double), cudaMemcpyHostToDevice));
    const Params p = params(h);
    const int grid = (h->n + 255) / 256;
    if (h->prec == LBM_F64)
        k_axi_init<double><<<grid, 256, 0, h->stream>>>(static_cast<double *>(h->f[h->parity]), p, h->rd);
    else
        k_axi_init<float><<<grid, 256, 0, h->stream>>>(static_cast<float *>(h->f[h->parity]), p, h->rd);
    ACK(h, cudaGetLastError());
    ACK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_axi_read_0d_state(lbm_axi_handle *h, int bc, double *out) {
    if (!h || !out || bc < 0 || bc >= (int)h->bcp.size()) return afail(h, LBM_ERR_ARG, "bad boundary");
    ACK(h, cudaSetDevice(h->device));
    ACK(h, cudaStreamSynchronize(h->stream));
    BcState s;
    ACK(h, cudaMemcpy(&s, h->bd.state + (size_t)(h->steps & 1) * h->bcp.size() + bc, sizeof s,
                      cudaMemcpyDeviceToHost));  // the slot written by the last step
    const BcParam &bp = h->bcp[bc];
    out[0] = (double)h->steps;
    out[1] = s.Q;
    out[2] = s.Qu;
    out[3] = s.Pbar - 1.0 / 3.0;
    out[4] = bp.kind == BC_RCR ? s.Pw : (bp.kind == BC_LV ? s.Pv : s.Pstar_gauge);
    out[5] = bp.kind == BC_LV ? s.Pv / h->etab_h[2 * (bp.etab_off + (int)(h->steps % bp.period))] : 0.0;
    out[6] = s.valve_open;
    out[7] = s.Td;
    return LBM_OK;
}

lbm_status lbm_axi_read_waveforms(lbm_axi_handle *h, double *out, int64_t max_rows, int64_t *rows) {
    if (!h || !out || !rows || max_rows < 0) return afail(h, LBM_ERR_ARG, "bad arguments");
    ACK(h, cudaSetDevice(h->device));
    ACK(h, cudaStreamSynchronize(h->stream));
    const int nb = (int)h->bcp.size();
    const int64_t have = nb ? std::min<int64_t>({h->steps, (int64_t)h->wave_cap, max_rows}) : 0;
    *rows = have;
    if (have == 0) return LBM_OK;
    const size_t width = 1 + 4 * (size_t)nb;
    std::vector<double> all((size_t)h->wave_cap * width);
    ACK(h, cudaMemcpy(all.data(), h->bd.wave, all.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t r = 0; r < have; r++) {
        const int64_t stepno = h->steps - have + r;
        memcpy(out + r * width, &all[(size_t)(stepno % h->wave_cap) * width], width * sizeof(double));
    }
    return LBM_OK;
}

const char *lbm_axi_last_error(const lbm_axi_handle *h) { return h ? h->err.c_str() : "null handle"; }

void lbm_axi_destroy(lbm_axi_handle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->s_bc) cudaStreamSynchronize(h->s_bc);
    if (h->ev_f) cudaEventDestroy(h->ev_f);
    if (h->ev_d) cudaEventDestroy(h->ev_d);
    if (h->s_bc) cudaStreamDestroy(h->s_bc);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (void *p : h->allocs) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
