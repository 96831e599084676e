// Device kernels of the per-step hot path besides the fused stream-collide
// (lbm_stream_collide.cu) and the immersed boundary (lbm_ib.cu):
//   k_bc_reduce       deterministic FP64 partial sums of the boundary flow Q
//                     and gauge pressure over the first fluid layer of each
//                     0D boundary (per-cell terms in the compute type), then,
//                     once per boundary, the FP64 forward-Euler 0D step (Eqs.
//                     rightbc, rightQ, LVE; valve switch and smoothing of
//                     Section 2.2.1)
//   k_bc_apply        the ghost populations of Eq. Non-equilibrium3 (per
//                     link, in the compute type)
//   k_gather          read-out of f(t_n), P and j for the host
//   k_wall_shear      wall shear stress at the fluid cells next to rigid walls
//   k_init, k_init_eq inverse of the pull: lays out a given f(t_0), or the
//                     equilibrium of given macroscopic fields
//   k_cycle_change    cycle-to-cycle change of the 0D waveforms
//
// Populations are stored as deviations s_i = f_i - w_i (FP32, FP16, BF16 or
// FP64) in structure-of-arrays order f[i][cell].  The resident state between
// steps is the post-collision field f*(t_n) with the ghost populations of
// the 0D boundary nodes for t_{n+1} already in their slots, so one step is:
// (immersed boundary) -> k_stream_collide -> k_bc_reduce -> k_bc_apply.
#include "lbm_device.cuh"
#include "lbm_zero_d.cuh"

namespace lbm {

__constant__ signed char c_ex[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ signed char c_ey[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ signed char c_ez[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

// ---------------------------------------------------------------------------
// 0D coupling.  The per-cell and per-link arithmetic runs in the compute type
// R of the populations (FP32 for FP32/FP16/BF16 storage: the FP64 pipe of
// this part is narrow), with pressures as deviations from P_ref = 1/3 so that
// FP32 keeps their resolution; the boundary sums and the 0D step are FP64.
template <class R>
__device__ __forceinline__ void forced_velocity(const KParams &p, int cf, R v[3]) {
    const size_t N = (size_t)p.n;
    const R *aux = static_cast<const R *>(p.aux);
    v[0] = aux[N + cf];
    v[1] = aux[2 * N + cf];
    v[2] = aux[3 * N + cf];
    if (__ldg(&p.flags[cf]) & FL_BAND) {
        const typename Vec4<R>::T bb = static_cast<const typename Vec4<R>::T *>(p.b)[cf];
        v[0] += R(0.5) * bb.x;
        v[1] += R(0.5) * bb.y;
        v[2] += R(0.5) * bb.z;
    }
}

// The 0D step of boundary b from the sums over its first layer (taken by one
// thread): the state of t_{n+1} and, if store, the state and the waveform row
// written; returns what the ghost pass needs.
static __device__ BcStepResult bc_step(const BcParam &P, int b, double Q, double Ps, long long n,
                                       const BcKParams &q, bool store) {
    const BcState old = q.state[(size_t)(n & 1) * q.n_bc_total + b];
    int ptype, closed;
    double Sm;
    const double Psum = (double)P.n_xf / 3.0 + Ps;  // sum of P over the layer
    const BcState st = zero_d_step(P, old, Q, Psum, (double)P.n_xf, n, q.etab, &ptype, &closed, &Sm);
    if (store) {
        q.state[(size_t)((n + 1) & 1) * q.n_bc_total + b] = st;
        double *w = q.wave + ((size_t)(n % q.wave_cap) * q.n_bc_total + b) * 4;
        w[0] = st.Qu;
        w[1] = st.Pbar - 1.0 / 3.0;
        w[2] = (P.kind == BC_RCR) ? st.Pw : (P.kind == BC_LV ? st.Pv : st.Pstar_gauge);
        w[3] = st.valve_open;
    }
    BcStepResult r;
    r.Pg = st.Pstar_gauge;
    r.S = Sm;
    r.cosp = r.sinp = 0.0;
    if (P.kind == BC_VELOCITY) {  // the inlet's phase, once for every link of the boundary
        const double wv = P.par[0], tn1 = (double)(n + 1);
        r.cosp = cos(wv * tn1);
        r.sinp = sin(wv * tn1);
    }
    r.ptype = ptype;
    r.closed = closed;
    r.pad0 = r.pad1 = 0;
    return r;
}

// The boundary's partial sums added by one warp in a fixed order (lane k
// takes partials k, k + 32, ..., then a butterfly), so that every caller gets
// the same bits.
static __device__ __forceinline__ void bc_sum_partials(const BcParam &P, const BcKParams &q, double *Q, double *Ps) {
    const int lane = threadIdx.x & 31;
    double a = 0.0, c = 0.0;
    for (int k = lane; k < P.n_red; k += 32) {
        a += __ldcg(&q.partial[2 * (P.red_off + k)]);
        c += __ldcg(&q.partial[2 * (P.red_off + k) + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    *Q = a;
    *Ps = c;
}

// Partial sums of the boundary flow Q = sum n.j / sum f and of the gauge
// pressure (P - P_ref = c_s^2 sum s) over one chunk of a boundary's first
// fluid layer (FP64 sums in a fixed tree order).  With q.step_in_reduce (many
// link blocks), the boundary's last chunk to arrive (a counter per boundary;
// no block waits for another) sums all partials and takes the 0D step once
// for the boundary; otherwise every link block of k_bc_apply takes it.
template <class R>
__global__ void __launch_bounds__(BC_CHUNK) k_bc_reduce(KParams p, BcKParams q) {
    const int b = q.red_bc[blockIdx.x], ch = q.red_chunk[blockIdx.x];
    const BcParam &P = q.par[b];
    const size_t N = (size_t)p.n;
    const R *aux = static_cast<const R *>(p.aux);
    const int a = ch * BC_CHUNK + threadIdx.x;
    __shared__ double sQ[BC_CHUNK], sP[BC_CHUNK];
    __shared__ int s_last;
    double Q = 0.0, Ps = 0.0;
    if (a < P.n_xf) {
        const int cf = q.xf[P.xf_off + a];
        const R sd = aux[cf];
        Q = (double)((R)P.sign * aux[(size_t)(1 + P.axis) * N + cf] / (R(1) + sd));
        Ps = (double)(sd / R(3));
    }
    sQ[threadIdx.x] = Q;
    sP[threadIdx.x] = Ps;
    __syncthreads();
    for (int s = BC_CHUNK / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sQ[threadIdx.x] += sQ[threadIdx.x + s];
            sP[threadIdx.x] += sP[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        q.partial[2 * (P.red_off + ch)] = sQ[0];
        q.partial[2 * (P.red_off + ch) + 1] = sP[0];
        if (q.step_in_reduce) {
            __threadfence();  // the partial is visible before the arrival is counted
            s_last = atomicAdd(&q.arrived[b], 1) == P.n_red - 1;
        }
    }
    if (!q.step_in_reduce) return;
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return;
    __threadfence();
    bc_sum_partials(P, q, &Q, &Ps);
    if (threadIdx.x != 0) return;
    q.arrived[b] = 0;  // for the next step (kernel boundaries order it)
    q.result[b] = bc_step(P, b, Q, Ps, *p.step, q, true);
}

// Ghost populations of one chunk of links, Eq. Non-equilibrium3 written as
//   f_i(x_b) = f*_i(x_f) + f^eq_i(P*, v*) - f^eq_i(P(x_f), v(x_f)),
// since f*_i(x_f) = f^eq_i + (1 - 1/tau) f^neq_i + F_i at x_f.
// STEP_HERE: the kernel for few link blocks, each of which takes the 0D step
// itself (the boundary's first chunk storing the state); otherwise the step's
// result comes from k_bc_reduce.  Two instances, so that the one without the
// step keeps its low register count.
template <class S, bool STEP_HERE>
__global__ void __launch_bounds__(BC_CHUNK) k_bc_apply(S *__restrict__ f, KParams p, BcKParams q) {
    using R = typename Storage<S>::R;
    const int b = q.app_bc[blockIdx.x], ch = q.app_chunk[blockIdx.x];
    const BcParam &P = q.par[b];
    const size_t N = (size_t)p.n;
    const R *aux = static_cast<const R *>(p.aux);
    const int L = ch * BC_CHUNK + threadIdx.x;
    const bool have = L < P.n_links;
    if (!STEP_HERE && !have) return;
    // the link's inputs, read before the 0D step's result is known (with
    // STEP_HERE they arrive while one thread takes the step): x_b, x_f and i,
    // the forced velocity, sum s and f*_i at x_f, and the closure velocity or
    // the inlet profile of the link's node
    int cb = 0, cf = 0, i = 0;
    R vf[3] = {R(0), R(0), R(0)}, sdf = R(0), post = R(0);
    double pr[3] = {0.0, 0.0, 0.0}, v0o[3] = {0.0, 0.0, 0.0};
    if (have) {
        cb = q.lk_xb[P.link_off + L];
        cf = q.lk_xf[P.link_off + L];
        i = q.lk_i[P.link_off + L];
        forced_velocity<R>(p, cf, vf);
        sdf = aux[cf];
        post = Storage<S>::ld(f + pidx(i, (uint32_t)cf, (uint32_t)N));
        if (P.kind == BC_VELOCITY) {
            const double *prof = q.profile + 3 * (size_t)(P.node_off + q.lk_node[P.link_off + L]);
            pr[0] = prof[0];
            pr[1] = prof[1];
            pr[2] = prof[2];
        } else if (P.kind == BC_LV) {  // v_0(T_d) of an earlier closure (rewritten below if one happens now)
            const double *v0 = q.v0 + 3 * (size_t)(P.xf_off + q.lk_xfi[P.link_off + L]);
            v0o[0] = v0[0];
            v0o[1] = v0[1];
            v0o[2] = v0[2];
        }
    }
    BcStepResult r;
    if (!STEP_HERE) {
        r = q.result[b];
    } else {
        __shared__ BcStepResult s_r;
        if (threadIdx.x < 32) {
            double Q, Ps;
            bc_sum_partials(P, q, &Q, &Ps);
            if (threadIdx.x == 0) s_r = bc_step(P, b, Q, Ps, *p.step, q, ch == 0);
        }
        __syncthreads();
        if (!have) return;
        r = s_r;
    }
    R dP, vs[3];  // P* - P(x_f) and v*
    if (r.ptype) {  // pressure-type: (P_0D(t_{n+1}), v(x_f, t_n))
        dP = (R)r.Pg - sdf / R(3);
        vs[0] = vf[0];
        vs[1] = vf[1];
        vs[2] = vf[2];
    } else {        // velocity-type: (P(x_f, t_n), v_0D(t_{n+1}))
        dP = R(0);
        vs[0] = vs[1] = vs[2] = R(0);
        if (P.kind == BC_VELOCITY) {
            vs[P.axis] = (R)((double)P.sign * (pr[0] + pr[1] * r.cosp - pr[2] * r.sinp));
        } else if (P.kind == BC_LV) {  // closed valve: v_0(T_d) S(t, T_d, N_S)
            R u0[3];
            if (r.closed) {  // v_0(T_d) = v(x_f, T_d); links sharing x_f store the same value
                double *v0 = q.v0 + 3 * (size_t)(P.xf_off + q.lk_xfi[P.link_off + L]);
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    u0[a] = vf[a];
                    v0[a] = (double)vf[a];
                }
            } else {
#pragma unroll
                for (int a = 0; a < 3; a++) u0[a] = (R)v0o[a];
            }
            const R Sm = (R)r.S;
            vs[0] = u0[0] * Sm;
            vs[1] = u0[1] * Sm;
            vs[2] = u0[2] * Sm;
        }
    }
    const R ex = c_ex[i], ey = c_ey[i], ez = c_ez[i];
    const R w = i == 0 ? R(1.0 / 3.0) : (i < 7 ? R(1.0 / 18.0) : R(1.0 / 36.0));
    const R eus = ex * vs[0] + ey * vs[1] + ez * vs[2];
    const R euf = ex * vf[0] + ey * vf[1] + ez * vf[2];
    const R us2 = vs[0] * vs[0] + vs[1] * vs[1] + vs[2] * vs[2];
    const R uf2 = vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2];
    const R dfeq = w * R(3) * dP + w * (R(3) * (eus - euf) + R(4.5) * (eus * eus - euf * euf) - R(1.5) * (us2 - uf2));
    Storage<S>::st(f + pidx(i, (uint32_t)cb, (uint32_t)N), post + dfeq);
}

// ---------------------------------------------------------------------------
// Read-out: f(t_n) = pull of the resident f*(t_{n-1}) (with ghosts), plus
// P = c_s^2 sum f and j = sum e f, for the cells [c0, c1) of one instance
// (outputs indexed c - c0 with stride M = c1 - c0; non-fluid cells get 0).
template <class S>
__global__ void k_gather(const S *__restrict__ fin, KParams p, int c0, int c1, double *fout19, double *mac4) {
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const uint32_t fl = p.flags[c];
    const size_t N = (size_t)p.n, M = (size_t)(c1 - c0), k = (size_t)(c - c0);
    if (!(fl & FL_ACTIVE)) {
        if (fout19)
            for (int i = 0; i < NQ; i++) fout19[i * M + k] = 0.0;
        for (int a = 0; a < 4; a++) mac4[a * M + k] = 0.0;
        return;
    }
    const int r = find_row(p, c);
    const int x = p.rows[r].x0 + (c - p.rows[r].off);
    double sum = 0, jx = 0, jy = 0, jz = 0;
    for (int i = 0; i < NQ; i++) {
        size_t idx;
        if (i == 0) idx = pidx(0, (uint32_t)c, (uint32_t)N);
        else if (fl & (1u << i)) idx = pidx(opp(i), (uint32_t)c, (uint32_t)N);
        else idx = pidx(i, (uint32_t)(p.rows[r].nb[nbk(i)] + x - cx(i)), (uint32_t)N);
        const double fi = (double)Storage<S>::ld(fin + idx) + wgt(i);
        if (fout19) fout19[i * M + k] = fi;
        sum += fi;
        jx += cx(i) * fi;
        jy += cy(i) * fi;
        jz += cz(i) * fi;
    }
    mac4[k] = sum / 3.0;
    mac4[M + k] = jx;
    mac4[2 * M + k] = jy;
    mac4[3 * M + k] = jz;
}

// Inverse of the pull: given f(t_0) at the fluid cells of [c0, c1), write
// every population into the slot it will be pulled from.
template <class S>
__global__ void k_init(S *__restrict__ fout, KParams p, const double *__restrict__ f19, int c0, int c1) {
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const uint32_t fl = p.flags[c];
    if (!(fl & FL_ACTIVE)) return;
    const size_t N = (size_t)p.n;
    const size_t M = (size_t)(c1 - c0);
    const int r = find_row(p, c);
    const int x = p.rows[r].x0 + (c - p.rows[r].off);
    for (int i = 0; i < NQ; i++) {
        const double s = f19[i * M + (c - c0)] - wgt(i);
        size_t idx;
        if (i == 0) idx = pidx(0, (uint32_t)c, (uint32_t)N);
        else if (fl & (1u << i)) idx = pidx(opp(i), (uint32_t)c, (uint32_t)N);
        else idx = pidx(i, (uint32_t)(p.rows[r].nb[nbk(i)] + x - cx(i)), (uint32_t)N);
        Storage<S>::st(fout + idx, (typename Storage<S>::R)s);
    }
}

// Wall shear stress at the fluid cells next to a rigid wall (the paper's
// case-study observable, WSS = mu dv_1/dx_3 there): viscous stress of f(t_n)
// from its non-equilibrium part, sigma = -(1 - 1/(2 tau)) [sum_i e_i e_i
// (f_i - f^eq_i) + (v b + b v)/2], traction on the wall normal n (the
// normalised sum of e_i over bounce-back directions, into the fluid), minus
// its normal part.  Output 3 doubles per cell of [c0, c1) (zero elsewhere).
template <class S>
__global__ void k_wall_shear(const S *__restrict__ fin, KParams p, int c0, int c1, double *out3) {
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const size_t N = (size_t)p.n, M = (size_t)(c1 - c0), k = (size_t)(c - c0);
    const uint32_t fl = p.flags[c];
    out3[k] = out3[M + k] = out3[2 * M + k] = 0.0;
    if (!(fl & FL_ACTIVE) || !(fl & FL_BBMASK)) return;
    const int r = find_row(p, c);
    const int x = p.rows[r].x0 + (c - p.rows[r].off);
    double f[NQ], sum = 0, jx = 0, jy = 0, jz = 0, n[3] = {0, 0, 0};
    for (int i = 0; i < NQ; i++) {
        size_t idx;
        if (i == 0) idx = pidx(0, (uint32_t)c, (uint32_t)N);
        else if (fl & (1u << i)) idx = pidx(opp(i), (uint32_t)c, (uint32_t)N);
        else idx = pidx(i, (uint32_t)(p.rows[r].nb[nbk(i)] + x - cx(i)), (uint32_t)N);
        f[i] = (double)Storage<S>::ld(fin + idx) + wgt(i);
        sum += f[i];
        jx += cx(i) * f[i];
        jy += cy(i) * f[i];
        jz += cz(i) * f[i];
        if (i > 0 && (fl & (1u << i))) {
            n[0] += cx(i);
            n[1] += cy(i);
            n[2] += cz(i);
        }
    }
    const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nn == 0.0) return;
    n[0] /= nn;
    n[1] /= nn;
    n[2] /= nn;
    double b[3] = {0, 0, 0};
    if (fl & FL_BAND) {
        using R = typename Storage<S>::R;
        const typename Vec4<R>::T bb = static_cast<const typename Vec4<R>::T *>(p.b)[c];
        b[0] = bb.x;
        b[1] = bb.y;
        b[2] = bb.z;
    }
    const double v[3] = {jx + 0.5 * b[0], jy + 0.5 * b[1], jz + 0.5 * b[2]};
    const double P = sum / 3.0, usq = 1.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < NQ; i++) {
        const double e[3] = {(double)cx(i), (double)cy(i), (double)cz(i)};
        const double eu = e[0] * v[0] + e[1] * v[1] + e[2] * v[2];
        const double fneq = f[i] - wgt(i) * (3.0 * P + 3.0 * eu + 4.5 * eu * eu - usq);
        for (int a = 0; a < 3; a++)
            for (int q = 0; q < 3; q++) pi[a][q] += e[a] * e[q] * fneq;
    }
    const double kf = -(1.0 - 0.5 * p.omega[p.rows[r].inst]);
    double t[3], tn = 0.0;
    for (int a = 0; a < 3; a++) {
        t[a] = 0.0;
        for (int q = 0; q < 3; q++) t[a] += kf * (pi[a][q] + 0.5 * (v[a] * b[q] + b[a] * v[q])) * n[q];
        tn += t[a] * n[a];
    }
    for (int a = 0; a < 3; a++) out3[a * M + k] = t[a] - tn * n[a];
}

// Equilibrium initialisation: f_i(x, t_0) = f^eq_i(P, v) (Eq. feq) from the
// macroscopic fields of the fluid cells of [c0, c1) (4 x M doubles: P, vx,
// vy, vz), laid out by the inverse of the pull like k_init.
template <class S>
__global__ void k_init_eq(S *__restrict__ fout, KParams p, const double *__restrict__ mac, int c0, int c1) {
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const uint32_t fl = p.flags[c];
    if (!(fl & FL_ACTIVE)) return;
    const size_t N = (size_t)p.n, M = (size_t)(c1 - c0), k = (size_t)(c - c0);
    const double P = mac[k], vx = mac[M + k], vy = mac[2 * M + k], vz = mac[3 * M + k];
    const double usq = 1.5 * (vx * vx + vy * vy + vz * vz);
    const int r = find_row(p, c);
    const int x = p.rows[r].x0 + (c - p.rows[r].off);
    for (int i = 0; i < NQ; i++) {
        const double eu = cx(i) * vx + cy(i) * vy + cz(i) * vz;
        const double s = wgt(i) * (3.0 * P - 1.0 + 3.0 * eu + 4.5 * eu * eu - usq);  // f^eq_i - w_i
        size_t idx;
        if (i == 0) idx = pidx(0, (uint32_t)c, (uint32_t)N);
        else if (fl & (1u << i)) idx = pidx(opp(i), (uint32_t)c, (uint32_t)N);
        else idx = pidx(i, (uint32_t)(p.rows[r].nb[nbk(i)] + x - cx(i)), (uint32_t)N);
        Storage<S>::st(fout + idx, (typename Storage<S>::R)s);
    }
}

// Cycle-to-cycle change of the boundary waveforms of one instance per CTA:
// over the last `period` recorded steps t, max over waveforms W in {Q_u, mean
// P} of each boundary of max_t |W(t) - W(t - period)| / max_t |W(t - period)|.
__global__ void k_cycle_change(BcKParams q, const int *bc_first, const int *n_bc, const long long *period,
                               long long steps, double *delta) {
    const int inst = blockIdx.x;
    const long long T = period[inst];
    if (T <= 0) {
        if (threadIdx.x == 0) delta[inst] = -1.0;
        return;
    }
    __shared__ double s_num[256], s_den[256];
    double worst = 0.0;
    for (int k = 0; k < n_bc[inst]; k++) {
        const int b = bc_first[inst] + k;
        for (int wv = 0; wv < 2; wv++) {
            double num = 0.0, den = 0.0;
            for (long long t = steps - T + threadIdx.x; t < steps; t += blockDim.x) {
                const double a = q.wave[((size_t)(t % q.wave_cap) * q.n_bc_total + b) * 4 + wv];
                const double c = q.wave[((size_t)((t - T) % q.wave_cap) * q.n_bc_total + b) * 4 + wv];
                num = fmax(num, fabs(a - c));
                den = fmax(den, fabs(c));
            }
            s_num[threadIdx.x] = num;
            s_den[threadIdx.x] = den;
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if (threadIdx.x < s) {
                    s_num[threadIdx.x] = fmax(s_num[threadIdx.x], s_num[threadIdx.x + s]);
                    s_den[threadIdx.x] = fmax(s_den[threadIdx.x], s_den[threadIdx.x + s]);
                }
                __syncthreads();
            }
            if (s_den[0] > 0.0) worst = fmax(worst, s_num[0] / s_den[0]);
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) delta[inst] = worst;
}

// ---------------------------------------------------------------------------
// launchers

cudaError_t launch_boundary(int prec, void *f, const KParams &p, const BcKParams &q, cudaStream_t s) {
    if (q.n_bc_total == 0) return cudaSuccess;
    if (prec == 3) k_bc_reduce<double><<<q.n_red_blocks, BC_CHUNK, 0, s>>>(p, q);
    else k_bc_reduce<float><<<q.n_red_blocks, BC_CHUNK, 0, s>>>(p, q);
    if (q.step_in_reduce) {
        DISPATCH(prec, (k_bc_apply<S, false><<<q.n_app_blocks, BC_CHUNK, 0, s>>>(as<S>(f), p, q)));
    } else {
        DISPATCH(prec, (k_bc_apply<S, true><<<q.n_app_blocks, BC_CHUNK, 0, s>>>(as<S>(f), p, q)));
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(int prec, const void *fin, const KParams &p, int c0, int c1, double *f19, double *mac4,
                          cudaStream_t s) {
    const int block = 256;
    const int grid = (c1 - c0 + block - 1) / block;
    if (grid == 0) return cudaSuccess;
    DISPATCH(prec, (k_gather<S><<<grid, block, 0, s>>>(static_cast<const S *>(fin), p, c0, c1, f19, mac4)));
    return cudaGetLastError();
}

// 0D state rows of boundaries [b0, b0 + nb) for lbm_read_0d_state_async:
// {t, Q, Q_u, Pbar_gauge, state, C_v P_v (LV), valve_open, T_d}
// the 8-value state row of boundary b after `steps` steps
__device__ __forceinline__ void state_row(const BcState *__restrict__ st, const BcParam *__restrict__ par,
                                          const double *__restrict__ etab, int b, int nbc_total, long long steps,
                                          double *o) {
    const BcState s = st[(size_t)(steps & 1) * nbc_total + b];
    const BcParam &P = par[b];
    o[0] = (double)steps;
    o[1] = s.Q;
    o[2] = s.Qu;
    o[3] = s.Pbar - 1.0 / 3.0;
    o[4] = P.kind == BC_RCR ? s.Pw : (P.kind == BC_LV ? s.Pv : s.Pstar_gauge);
    o[5] = P.kind == BC_LV ? s.Pv / etab[2 * (P.etab_off + (int)(steps % P.period))] : 0.0;
    o[6] = s.valve_open;
    o[7] = s.Td;
}

__global__ void k_state_rows(const BcState *__restrict__ st, const BcParam *__restrict__ par,
                             const double *__restrict__ etab, int b0, int nb, int nbc_total, long long steps,
                             double *out8) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    state_row(st, par, etab, b0 + k, nbc_total, steps, out8 + 8 * (size_t)k);
}

// Per-step 0D input and output of lbm_step_io, in stream order around each
// step.  *cursor counts the call's steps taken so far.  k_io_params copies the
// np params of step *cursor (from page-locked host memory that the device
// addresses) into the boundary's device parameters; k_io_state writes the
// state rows of nb boundaries after the step (step count *step + 1, the step
// index t_n of the step just taken plus one) to out8 + 8 nb *cursor and then
// advances *cursor.
__global__ void k_io_params(const double *__restrict__ params, int np, BcParam *par, const long long *cursor) {
    const long long c = *cursor;
    if ((int)threadIdx.x < np) par->par[threadIdx.x] = params[c * np + threadIdx.x];
}

__global__ void k_io_state(const BcState *__restrict__ st, const BcParam *__restrict__ par,
                           const double *__restrict__ etab, int b0, int nb, int nbc_total,
                           const long long *__restrict__ step, double *out8, long long *cursor) {
    const long long c = *cursor;
    const int k = threadIdx.x;
    if (k < nb) state_row(st, par, etab, b0 + k, nbc_total, *step + 1, out8 + 8 * ((size_t)c * nb + k));
    __syncthreads();
    if (threadIdx.x == 0) *cursor = c + 1;
}

cudaError_t launch_io_params(const double *params, int np, BcParam *par, const long long *cursor, cudaStream_t s) {
    k_io_params<<<1, 32, 0, s>>>(params, np, par, cursor);
    return cudaGetLastError();
}

cudaError_t launch_io_state(const BcState *st, const BcParam *par, const double *etab, int b0, int nb, int nbc_total,
                            const long long *step, double *out8, long long *cursor, cudaStream_t s) {
    k_io_state<<<1, 32 * ((nb + 31) / 32), 0, s>>>(st, par, etab, b0, nb, nbc_total, step, out8, cursor);
    return cudaGetLastError();
}

cudaError_t launch_state_rows(const BcState *st, const BcParam *par, const double *etab, int b0, int nb,
                              int nbc_total, long long steps, double *out8, cudaStream_t s) {
    if (nb == 0) return cudaSuccess;
    k_state_rows<<<1, 32 * ((nb + 31) / 32), 0, s>>>(st, par, etab, b0, nb, nbc_total, steps, out8);
    return cudaGetLastError();
}

// Small stream-ordered transfer in 8-byte words, between mapped page-locked
// host memory and device memory, on the compute engine (no hand-off to a
// copy engine and back).
__global__ void k_copy_words(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst,
                             int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

cudaError_t launch_copy_words(const void *src, void *dst, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    if (bytes % 8 != 0) return cudaErrorInvalidValue;
    k_copy_words<<<1, 32, 0, s>>>(static_cast<const unsigned long long *>(src), static_cast<unsigned long long *>(dst),
                                  (int)(bytes / 8));
    return cudaGetLastError();
}

// compact -> box scatter of the gathered P, j into FP32 device arrays
__global__ void k_scatter_box(const double *__restrict__ mac4, int M, const int32_t *__restrict__ box, float *P,
                              float *jx, float *jy, float *jz) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int b = box[m];
    P[b] = (float)mac4[m];
    jx[b] = (float)mac4[M + m];
    jy[b] = (float)mac4[2 * (size_t)M + m];
    jz[b] = (float)mac4[3 * (size_t)M + m];
}

cudaError_t launch_scatter_box(const double *mac4, int M, const int32_t *box, float *P, float *jx, float *jy,
                               float *jz, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    k_scatter_box<<<(M + 255) / 256, 256, 0, s>>>(mac4, M, box, P, jx, jy, jz);
    return cudaGetLastError();
}

cudaError_t launch_wall_shear(int prec, const void *fin, const KParams &p, int c0, int c1, double *out3,
                              cudaStream_t s) {
    const int block = 128;
    const int grid = (c1 - c0 + block - 1) / block;
    if (grid == 0) return cudaSuccess;
    DISPATCH(prec, (k_wall_shear<S><<<grid, block, 0, s>>>(static_cast<const S *>(fin), p, c0, c1, out3)));
    return cudaGetLastError();
}

cudaError_t launch_init_eq(int prec, void *fout, const KParams &p, const double *mac, int c0, int c1,
                           cudaStream_t s) {
    const int block = 256;
    const int grid = (c1 - c0 + block - 1) / block;
    if (grid == 0) return cudaSuccess;
    DISPATCH(prec, (k_init_eq<S><<<grid, block, 0, s>>>(as<S>(fout), p, mac, c0, c1)));
    return cudaGetLastError();
}

cudaError_t launch_cycle_change(const BcKParams &q, const int *bc_first, const int *n_bc, const long long *period,
                                long long steps, double *delta, int n_inst, cudaStream_t s) {
    k_cycle_change<<<n_inst, 256, 0, s>>>(q, bc_first, n_bc, period, steps, delta);
    return cudaGetLastError();
}

cudaError_t launch_init(int prec, void *fout, const KParams &p, const double *f19, int c0, int c1,
                        cudaStream_t s) {
    const int block = 256;
    const int grid = (c1 - c0 + block - 1) / block;
    if (grid == 0) return cudaSuccess;
    DISPATCH(prec, (k_init<S><<<grid, block, 0, s>>>(as<S>(fout), p, f19, c0, c1)));
    return cudaGetLastError();
}

}  // namespace lbm
