// Fused stream-collide kernel (one launch per time step over every stored
// cell of every instance) and its launcher with the autotuner's variants.
#include "lbm_device.cuh"

namespace lbm {

// One base pointer per direction of the input and output population arrays
// (f_i = f + i N, structure of arrays), passed in the kernel's parameter
// space: every pull and store then forms its address with one wide
// multiply-add from a constant-bank operand.
template <class S> struct PopDirs {
    const S *in[NQ];
    S *out[NQ];
};

// ---------------------------------------------------------------------------
// Fused stream-collide.  For each fluid cell x and direction i the pulled
// population is f*_i(x - e_i) (or f*_opp(i)(x) when x - e_i is a rigid wall:
// halfway bounce-back).  Then P = c_s^2 sum f, j = sum e f, v = j + b/2
// (Eqs. rho, v), f^eq (Eq. feq), the forcing F_i (Eq. f) and BGK relaxation
// (Eq. fi).  With s = f - w: sum f = 1 + sum s, j = sum e s, and
// f^eq_i - w_i = w_i (K + 3 e.v + 9/2 (e.v)^2), K = sum s - 3/2 v^2.
//
// Arithmetic per cell, arranged for few instructions (the 16-bit storage
// variants are bound by instruction issue, not by bytes):
// * pull: the pull source of direction i lies on one of 8 neighbouring
//   lattice lines (or the own row), at x - e_ix; a bounce-back link instead
//   reads the opposite population of the own cell, which in this layout is
//   f_i + (opp(i) - i) N + c with opp(i) - i = +-1, so one select of a
//   32-bit index per direction covers both cases;
// * moments from the sums and differences of the 9 opposite pairs;
// * relaxation per opposite pair (i, i'): with A = omega w (K + 9/2 (e.v)^2)
//   and B = 3 omega w e.v, s*_i = (1 - omega) s_i + A + B and
//   s*_i' = (1 - omega) s_i' + A - B; Guo's F_i splits the same way into the
//   pair-symmetric part w (1 - omega/2) (9 (e.v)(e.b) - 3 v.b) and the
//   antisymmetric 3 w (1 - omega/2) e.b.  The forcing is evaluated only by
//   warps that hold a band cell (a warp-uniform branch).
//
// Occupancy request to ptxas (template parameter MINB: at least MINB resident
// 256-thread blocks per SM).  CPT > 1 gives each thread CPT independent
// cells, one grid stride apart, whose loads are all issued before any of
// them is consumed.  The variants are kept for the run-time autotuner.
// desc = 1 maps the blocks to the cells in descending order, so that a
// launch starts on the lines the previous kernel touched last (still in L2).
template <class S, class R, bool FORCED>
__device__ __forceinline__ void collide_store(const PopDirs<S> &d, const KParams &p, const R (&f)[NQ], R omega,
                                              uint32_t fl, int c) {
    constexpr int NP = (NQ - 1) / 2;
    R Sp[NP], Dp[NP];
#pragma unroll
    for (int q = 0; q < NP; q++) {
        Sp[q] = f[2 * q + 1] + f[2 * q + 2];
        Dp[q] = f[2 * q + 1] - f[2 * q + 2];
    }
    R sd = f[0], jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < NP; q++) {
        sd += Sp[q];
        const int i = 2 * q + 1;
        if (cx(i) > 0) jx += Dp[q];
        if (cx(i) < 0) jx -= Dp[q];
        if (cy(i) > 0) jy += Dp[q];
        if (cy(i) < 0) jy -= Dp[q];
        if (cz(i) > 0) jz += Dp[q];
        if (cz(i) < 0) jz -= Dp[q];
    }
    R bx = 0, by = 0, bz = 0;
    if (FORCED && (fl & FL_BAND)) {
        const typename Vec4<R>::T bb = static_cast<const typename Vec4<R>::T *>(p.b)[c];
        bx = bb.x;
        by = bb.y;
        bz = bb.z;
    }
    const R vx = FORCED ? jx + R(0.5) * bx : jx;
    const R vy = FORCED ? jy + R(0.5) * by : jy;
    const R vz = FORCED ? jz + R(0.5) * bz : jz;
    if (fl & FL_XF) {
        R *aux = static_cast<R *>(p.aux);
        const size_t N = (size_t)p.n;
        aux[c] = sd;
        aux[N + c] = jx;
        aux[2 * N + c] = jy;
        aux[3 * N + c] = jz;
    }
    const R vv = vx * vx + vy * vy + vz * vz;
    if (!(sd - sd == R(0)) || !(vv <= R(0.09))) atomicOr(p.status, 1u);

    const R om1 = R(1) - omega;
    const R K = sd - R(1.5) * vv;
    // per weight class (1/18 faces, 1/36 edges): omega w K, 9/2 omega w, 3 omega w
    const R ow1 = omega * R(1.0 / 18.0), ow2 = omega * R(1.0 / 36.0);
    const R wK1 = ow1 * K, wK2 = ow2 * K;
    const R a1 = R(4.5) * ow1, a2 = R(4.5) * ow2;
    const R b1 = R(3) * ow1, b2 = R(3) * ow2;
    R kw1 = 0, kw2 = 0, vb = 0;
    if (FORCED) {
        const R kf = R(1) - R(0.5) * omega;
        kw1 = kf * R(1.0 / 18.0);
        kw2 = kf * R(1.0 / 36.0);
        vb = vx * bx + vy * by + vz * bz;
    }
    R post0 = om1 * f[0] + omega * R(1.0 / 3.0) * K;
    if (FORCED) post0 -= (R(1) - R(0.5) * omega) * vb;  // w_0 (1 - omega/2) (-3 v.b), w_0 = 1/3
    Storage<S>::st(d.out[0] + c, post0);
#pragma unroll
    for (int q = 0; q < NP; q++) {
        const int i = 2 * q + 1;
        const bool face = i < 7;
        R eu = 0, eb = 0;
        if (cx(i) > 0) eu += vx;
        if (cx(i) < 0) eu -= vx;
        if (cy(i) > 0) eu += vy;
        if (cy(i) < 0) eu -= vy;
        if (cz(i) > 0) eu += vz;
        if (cz(i) < 0) eu -= vz;
        R A = (face ? a1 : a2) * eu * eu + (face ? wK1 : wK2);
        R B = (face ? b1 : b2) * eu;
        if (FORCED) {
            if (cx(i) > 0) eb += bx;
            if (cx(i) < 0) eb -= bx;
            if (cy(i) > 0) eb += by;
            if (cy(i) < 0) eb -= by;
            if (cz(i) > 0) eb += bz;
            if (cz(i) < 0) eb -= bz;
            const R kw = face ? kw1 : kw2;
            A += kw * (R(9) * eu * eb - R(3) * vb);
            B += R(3) * kw * eb;
        }
        Storage<S>::st(d.out[i] + c, om1 * f[i] + (A + B));
        Storage<S>::st(d.out[i + 1] + c, om1 * f[i + 1] + (A - B));
    }
}

// The launch covers the stored cells [c0, c1); the launch with bump = 1
// advances the step counter.
template <class S, int MINB, int CPT>
__global__ void __launch_bounds__(256, MINB)
    k_stream_collide(const __grid_constant__ PopDirs<S> d, const __grid_constant__ KParams p, int desc, int c0,
                     int c1, int bump) {
    using R = typename Storage<S>::R;
    const int bid = desc ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int t = c0 + bid * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (bump && t == c0 && p.step) *p.step += 1;  // the step index t_n seen by the boundary kernels
    const int N = (int)p.n;  // 19 N < 2^31 is checked at creation
    R f[CPT][NQ];
    R om[CPT];
    uint32_t fl[CPT];
#pragma unroll
    for (int u = 0; u < CPT; u++) {
        const int c = t + u * stride;
        fl[u] = c < c1 ? __ldg(&p.flags[c]) : 0u;
        om[u] = R(0);
        if (!(fl[u] & FL_ACTIVE)) continue;
        const int r = find_row(p, c);
        const int4 *row = reinterpret_cast<const int4 *>(p.rows + r);
        const int4 h0 = __ldg(row), h1 = __ldg(row + 1), h2 = __ldg(row + 2), h3 = __ldg(row + 3);
        // h0 = {off, x0, len, inst}, h1 = {y, z, nb0, nb1}, h2 = {nb2..nb5}, h3 = {nb6, nb7, nb8, pad}
        om[u] = omega_of<R>(p, h0.w);
        const int x = h0.y + (c - h0.x);
        const int line[9] = {h1.z + x, h1.w + x, h2.x + x, h2.y + x, c, h2.w + x, h3.x + x, h3.y + x, h3.z + x};
        f[u][0] = Storage<S>::ld(d.in[0] + c);
#pragma unroll
        for (int i = 1; i < NQ; i++) {
            const int src = line[nbk(i)] - cx(i);               // pull from x - e_i
            const int own = c + ((i & 1) ? N : -N);              // f_opp(i)(x) = f_i + (opp(i) - i) N + x
            const int idx = ((fl[u] >> i) & 1u) ? own : src;     // halfway bounce-back
            f[u][i] = Storage<S>::ld(d.in[i] + idx);
        }
    }
#pragma unroll
    for (int u = 0; u < CPT; u++) {
        const int c = t + u * stride;
        const bool band = (fl[u] & (FL_ACTIVE | FL_BAND)) == (FL_ACTIVE | FL_BAND);
        if (__any_sync(0xffffffffu, band)) {
            if (fl[u] & FL_ACTIVE) collide_store<S, R, true>(d, p, f[u], om[u], fl[u], c);
        } else {
            if (fl[u] & FL_ACTIVE) collide_store<S, R, false>(d, p, f[u], om[u], fl[u], c);
        }
    }
}

// ---------------------------------------------------------------------------
// launcher

// variants: {min blocks per SM, cells per thread}
static const int kVariants[SC_VARIANTS][2] = {{6, 1}, {8, 1}, {5, 1}, {4, 2}, {3, 2}};

int stream_collide_min_blocks(int variant) { return kVariants[variant][0]; }
int stream_collide_cells_per_thread(int variant) { return kVariants[variant][1]; }

template <class S> static PopDirs<S> pop_dirs(const void *fin, void *fout, long long n) {
    PopDirs<S> d;
    for (int i = 0; i < NQ; i++) {
        d.in[i] = static_cast<const S *>(fin) + (size_t)i * (size_t)n;
        d.out[i] = static_cast<S *>(fout) + (size_t)i * (size_t)n;
    }
    return d;
}

cudaError_t launch_stream_collide(int prec, const void *fin, void *fout, const KParams &p, int block,
                                  int variant, cudaStream_t s, int desc, int c0, int c1, int bump) {
    if (c1 < 0) c1 = (int)p.n;
    if (c1 <= c0) return cudaSuccess;
    if (block % 32) return cudaErrorInvalidValue;  // whole warps: the forcing branch is a warp vote
    const int cpt = kVariants[variant][1];
    const int grid = (int)((c1 - c0 + (long long)block * cpt - 1) / ((long long)block * cpt));
    switch (variant) {
    case 1:
        DISPATCH(prec, (k_stream_collide<S, 8, 1><<<grid, block, 0, s>>>(pop_dirs<S>(fin, fout, p.n), p, desc, c0, c1, bump)));
        break;
    case 2:
        DISPATCH(prec, (k_stream_collide<S, 5, 1><<<grid, block, 0, s>>>(pop_dirs<S>(fin, fout, p.n), p, desc, c0, c1, bump)));
        break;
    case 3:
        DISPATCH(prec, (k_stream_collide<S, 4, 2><<<grid, block, 0, s>>>(pop_dirs<S>(fin, fout, p.n), p, desc, c0, c1, bump)));
        break;
    case 4:
        DISPATCH(prec, (k_stream_collide<S, 3, 2><<<grid, block, 0, s>>>(pop_dirs<S>(fin, fout, p.n), p, desc, c0, c1, bump)));
        break;
    default:
        DISPATCH(prec, (k_stream_collide<S, 6, 1><<<grid, block, 0, s>>>(pop_dirs<S>(fin, fout, p.n), p, desc, c0, c1, bump)));
        break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
