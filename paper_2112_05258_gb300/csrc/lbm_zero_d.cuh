// The 0D models of the coupled boundaries on the device (FP64): the
// smoothing function, the ODE right-hand sides and one marching step with
// the valve logic of the hybrid LV inlet.  Shared by the 3D and the
// axisymmetric boundary kernels.
#pragma once
#include "lbm_kernels.h"

namespace lbm {

static __device__ __forceinline__ double smooth_to_zero(double t, double t0, double LS) {
    // Eq. SmoothFunction
    if (t < t0) return 1.0;
    if (t > t0 + LS) return 0.0;
    const double u = (t - t0) / LS;
    if (u <= 0.0) return 1.0;
    if (u >= 1.0) return 0.0;
    return exp(2.0 * exp(-1.0 / u) / (u - 1.0));
}

// Right-hand sides of the 0D ODEs with the boundary flow held over the step:
// Windkessel chamber (Eqs. rightbc, rightQ with P eliminated) and ventricle
// (Eq. LVE with C_v = 1/E: dP_v/dt = (E'/E) P_v - E Q).
static __device__ __forceinline__ double rcr_rate(double Pw, double Qout, double C, double Rd) {
    return Qout / C - Pw / (Rd * C);
}
static __device__ __forceinline__ double lv_rate(double Pv, double E, double Ed, double Q) { return (Ed / E) * Pv - E * Q; }

// Elastance between table steps n and n+1 at s in [0, 1] by cubic Hermite
// interpolation of the tabulated (E, dE/dt) at both ends.
static __device__ __forceinline__ void hermite_elastance(double E0, double D0, double E1, double D1, double s, double *E,
                                                  double *D) {
    const double s2 = s * s, s3 = s2 * s;
    *E = (2 * s3 - 3 * s2 + 1) * E0 + (s3 - 2 * s2 + s) * D0 + (-2 * s3 + 3 * s2) * E1 + (s3 - s2) * D1;
    *D = (6 * s2 - 6 * s) * E0 + (3 * s2 - 4 * s + 1) * D0 + (-6 * s2 + 6 * s) * E1 + (3 * s2 - 2 * s) * D1;
}

// The 0D step of one boundary from its state at t_n, given Q(t_n), the
// layer's pressure sum and its area (node count in 3D, sum of 2 pi r in the
// axisymmetric model).  Returns the state at t_{n+1}.  par[4] selects the
// marching scheme: 0 or 1 forward Euler (the paper's), 2 Heun, 4 classical
// Runge-Kutta (the paper allows higher order).  The forward-Euler forms are
// written exactly as before so that the default trajectory is unchanged.
static __device__ BcState zero_d_step(const BcParam &P, const BcState &old, double Qt, double Psum, double area,
                                      long long n, const double *etab, int *ptype, int *closed, double *Smooth) {
    const double PREF = 1.0 / 3.0;
    BcState st = old;
    st.Q = Qt;
    st.Qu = P.q_scale ? Qt / area : Qt;
    st.Pbar = Psum / area;
    *ptype = 1;
    *closed = 0;
    *Smooth = 0.0;
    const int order = (int)P.par[4];
    if (P.kind == BC_RCR) {
        // Eqs. rightbc/rightQ driven by the outflow -Q_u
        const double Qout = -st.Qu, C = P.par[1], Rd = P.par[2], P0 = old.Pw;
        double Pw;
        if (order == 2) {
            const double k1 = rcr_rate(P0, Qout, C, Rd), k2 = rcr_rate(P0 + k1, Qout, C, Rd);
            Pw = P0 + 0.5 * (k1 + k2);
        } else if (order == 4) {
            const double k1 = rcr_rate(P0, Qout, C, Rd), k2 = rcr_rate(P0 + 0.5 * k1, Qout, C, Rd);
            const double k3 = rcr_rate(P0 + 0.5 * k2, Qout, C, Rd), k4 = rcr_rate(P0 + k3, Qout, C, Rd);
            Pw = P0 + (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
        } else {
            Pw = P0 + (Qout / C - P0 / (Rd * C));
        }
        st.Pw = Pw;
        st.Pstar_gauge = Pw + P.par[0] * Qout;
    } else if (P.kind == BC_PRESSURE) {
        st.Pstar_gauge = P.par[0];
    } else if (P.kind == BC_LV) {
        // Eq. LVE with C_v = 1/E: P_v <- P_v - (1/C_v)(dC_v/dt P_v + Q), dC_v/dt = -E'/E^2
        const int T = P.period;
        const double E = etab[2 * (P.etab_off + (int)(n % T))];
        const double Ed = etab[2 * (P.etab_off + (int)(n % T)) + 1];
        const double Qin = (old.valve_open != 0.0) ? st.Qu : 0.0;
        double Pv;
        if (order == 2 || order == 4) {
            const double E1 = etab[2 * (P.etab_off + (int)((n + 1) % T))];
            const double D1 = etab[2 * (P.etab_off + (int)((n + 1) % T)) + 1];
            const double P0 = old.Pv;
            if (order == 2) {
                const double k1 = lv_rate(P0, E, Ed, Qin), k2 = lv_rate(P0 + k1, E1, D1, Qin);
                Pv = P0 + 0.5 * (k1 + k2);
            } else {
                double Eh, Dh;
                hermite_elastance(E, Ed, E1, D1, 0.5, &Eh, &Dh);
                const double k1 = lv_rate(P0, E, Ed, Qin), k2 = lv_rate(P0 + 0.5 * k1, Eh, Dh, Qin);
                const double k3 = lv_rate(P0 + 0.5 * k2, Eh, Dh, Qin), k4 = lv_rate(P0 + k3, E1, D1, Qin);
                Pv = P0 + (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
            }
        } else {
            const double Cv = 1.0 / E, dCv = -Ed / (E * E);
            Pv = old.Pv - (1.0 / Cv) * (dCv * old.Pv + Qin);
        }
        if (old.valve_open != 0.0) {
            if (st.Qu < 0.0) {  // closure: the inflow has reversed
                st.valve_open = 0.0;
                st.Td = (double)n;
                *closed = 1;
            }
        } else {
            if (Pv < P.par[1]) Pv = P.par[1];           // ideal mitral diode from P_la
            if (Pv > st.Pbar - PREF) st.valve_open = 1.0;  // ventricle exceeds the inlet pressure
        }
        st.Pv = Pv;
        st.Pstar_gauge = Pv;
        *ptype = st.valve_open != 0.0;
        *Smooth = smooth_to_zero((double)(n + 1), st.Td, P.par[2]);
    } else {
        *ptype = 0;
    }
    return st;
}

}  // namespace lbm
