/*
 * liblbm -- axisymmetric lattice: the 3D-axisymmetric D2Q9 model of
 * Section 2.3.1 (Eq. Afi: BGK with forcing and the axisymmetric source H_i)
 * coupled to the same 0D boundaries as the 3D lattice (Section 2.2).
 *
 * Coordinates are pseudo-Cartesian (x, r) with node (x, j) at r = j + 1/2
 * (lattice units, dx = dt = 1); the symmetry axis r = 0 lies below row 0 and
 * acts as a mirror.  Node codes: 0 fluid, 1 rigid wall (halfway
 * bounce-back), 2 + k node of 0D boundary k, which must be a column at
 * x = 0 (sign +1) or x = nx - 1 (sign -1) with axis 0.  Rows above nr - 1
 * and columns outside [0, nx) are walls.
 *
 * The source terms follow from the axisymmetric incompressible equations
 * (the printed h^(2) of Eq. AH1 is not legible): mass source m = -u_r / r,
 * S_i = (1 - 1/(2 tau)) w_i m with P = c_s^2 (sum f + m/2), and the momentum
 * corrections g_x = nu (d_r u_x + d_x u_r)/r - u_x u_r / r,
 * g_r = 2 nu (d_r u_r - u_r / r)/r - u_r^2 / r through the Guo term, the
 * strain rates taken from the local non-equilibrium stress.  The boundary
 * flow of a 0D boundary is Q = sum over its first fluid layer of
 * 2 pi r n.j / sum f (area 2 pi r per node), Q_u = Q / A; its pressure the
 * area-weighted mean.
 *
 * Errors: LBM_ERR_ARG (nothing done), LBM_ERR_CUDA (see lbm_axi_last_error),
 * LBM_ERR_UNSTABLE from lbm_axi_sync when a NaN/Inf or |v| > 0.3 was seen.
 */
#ifndef LBM_AXI_H
#define LBM_AXI_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, nr;
    const uint8_t *node;          /* host, nr x nx codes, x fastest (copied) */
    double tau;                   /* > 0.5 */
    int q_scale;                  /* 1: 0D models see Q_u = Q / A; 0: Q */
    int n_bc;                     /* <= 8 */
    const lbm_boundary_desc *bc;  /* kinds and params as in lbm.h; axis 0 */
    int precision;                /* LBM_F32 or LBM_F64 */
    void *stream;                 /* cudaStream_t to enqueue on; NULL: the library creates one */
    int device;
    int graph_steps;              /* steps per captured CUDA graph (even); 0 = 64 */
    int wave_capacity;            /* waveform ring buffer in steps; 0 = 8192 */
} lbm_axi_config;

typedef struct lbm_axi_handle lbm_axi_handle;

/* Builds the lattice at rest (f_i = w_i) with the 0D states from params. */
lbm_status lbm_axi_create(const lbm_axi_config *cfg, lbm_axi_handle **out);

/* Advances n steps (Algorithm 1 with Eq. Afi); asynchronous. */
lbm_status lbm_axi_step(lbm_axi_handle *h, int64_t n);

/* Waits for the stream; LBM_ERR_UNSTABLE if the device status word is set. */
lbm_status lbm_axi_sync(lbm_axi_handle *h);

/* Host outputs, nr x nx doubles each (zero off the fluid): P = c_s^2
 * (sum f + m/2) and the fluid velocity j + g/2 of f(t_n). */
lbm_status lbm_axi_read_fields(lbm_axi_handle *h, double *P, double *ux, double *ur);

/* Host output: f_i(x, t_n) as 9 x (nr*nx) doubles (non-fluid 0); the D2Q9
 * order is e = (0,0), (1,0), (-1,0), (0,1), (0,-1), (1,1), (-1,-1), (1,-1),
 * (-1,1) in (e_x, e_r). */
lbm_status lbm_axi_read_populations(lbm_axi_handle *h, double *f);

/* Sets f_i(x, t_0) at every fluid node from 9 x (nr*nx) host doubles. */
lbm_status lbm_axi_init_populations(lbm_axi_handle *h, const double *f);

/* 8 doubles per boundary as lbm_read_0d_state. */
lbm_status lbm_axi_read_0d_state(lbm_axi_handle *h, int bc, double *out);

/* Rows of 1 + 4 n_bc doubles as lbm_read_waveforms. */
lbm_status lbm_axi_read_waveforms(lbm_axi_handle *h, double *out, int64_t max_rows, int64_t *rows);

const char *lbm_axi_last_error(const lbm_axi_handle *h);
void lbm_axi_destroy(lbm_axi_handle *h);

#ifdef __cplusplus
}
#endif
#endif
