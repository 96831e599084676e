// Kernel parameter blocks and launchers (internal to liblbm).
#pragma once
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// Four-component vectors of the compute type, one per cell (array of structures),
// so that a cell's force or velocity is one vector load and one vector atomic.
template <class R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
struct alignas(32) double4a { double x, y, z, w; };
template <> struct Vec4<double> { using T = double4a; };

// Lattice-wide pointers shared by the kernels (device memory).
struct KParams {
    long long n;                // stored cells = population stride
    const uint32_t *flags;      // per cell
    const RowInfo *rows;        // rows + sentinel
    const int32_t *chunk_row;   // per 32-cell chunk: {row of its first cell, new-row lane mask}
    const double *omega;        // per instance, 1/tau
    const float *omega_f;       // the same rounded to FP32 (no FP64 conversion per cell)
    const void *b;              // force density b, 4 x compute type per cell (x, y, z, unused)
    void *aux;                  // first-layer macros (sum s, jx, jy, jz), compute type, 4 x n
    long long *step;            // index t_n of the step in progress
    unsigned *status;           // bit 0: NaN/Inf or |v| > 0.3 seen
};

// 0D boundary tables (device memory).  The boundary work of a step runs as
// two kernels: k_bc_reduce (one CTA per chunk of BC_CHUNK first-layer cells
// writes an FP64 partial sum) and k_bc_apply (one CTA per chunk of BC_CHUNK
// links writes the ghosts).  The 0D step from the state of t_n (the partials
// summed in a fixed order) is taken either by the boundary's last reduce CTA
// to finish, which stores the state of t_{n+1} and the step's result, or,
// when the link CTAs fit in one wave, by every link CTA (the boundary's first
// one storing the state): the same arithmetic either way.
struct BcStepResult {
    double Pg;          // P* - P_ref of a pressure-type coupling
    double S;           // smoothing factor S(t_{n+1}) of a closed LV valve
    double cosp, sinp;  // velocity inlet: cos and sin of omega t_{n+1}
    int ptype;          // 1: pressure-type ghosts, 0: velocity-type
    int closed;         // 1: the LV valve closed in this step
    int pad0, pad1;
};
struct BcKParams {
    int n_bc_total;
    const BcParam *par;
    BcState *state;             // [2][n_bc_total]: step n reads state[n & 1], writes state[(n + 1) & 1]
    const int32_t *xf;
    const int32_t *lk_xb, *lk_xf, *lk_node, *lk_xfi;
    const uint8_t *lk_i;
    const double *profile;
    const double *etab;
    double *v0;                 // 3 per first-layer entry
    double *wave;               // ring buffer [cap][n_bc_total][4]
    int wave_cap;
    double *partial;            // 2 per reduce chunk: sum n.j/sum f, sum (P - P_ref)
    int step_in_reduce;         // 1: the 0D step once per boundary in k_bc_reduce; 0: in every k_bc_apply block
    int *arrived;               // per boundary: reduce CTAs done in this step (back to 0 after it)
    BcStepResult *result;       // per boundary
    int n_red_blocks, n_app_blocks;
    const int32_t *red_bc, *red_chunk;  // per reduce block
    const int32_t *app_bc, *app_chunk;  // per apply block
};

// Immersed-boundary tables (device memory).
struct IbKParams {
    int n_nodes;                // all instances
    int n_band;
    const int32_t *band;        // compact band cells
    const int32_t *node_inst;   // per node
    const InstParam *inst;
    const int32_t *rowid;
    // wall-node state, 3 per node: FP64 with FP64 storage (X, V_s, I, F, V_f);
    // FP32 otherwise, with the position as the displacement D = X - X0
    double *X, *Vs, *I, *F, *Vf;
    float *D32, *Vs32, *I32, *F32, *Vf32;
    const double *X0, *dA, *ks;
    const float *g0, *dA32, *ks32;  // X0 - 1/2 - ref (3 per node), dA, k_s in FP32
    const uint8_t *pinned;
    void *vband;                // fluid velocity j + b/2 (previous step's b) at band cells, 4 x compute type per cell
    int threads_per_node;       // 1, 2 or 4 threads of the node kernel per wall node
    const int32_t *order;       // wall nodes grouped by slab (null: index order)
    const int32_t *lines;       // 36 per node: compact index of x = 0 on the support lines
    const uint64_t *mask;       // 4 per node: fluid cells of the 6^3 box around the reference cell
    const int32_t *ref;         // 3 per node: reference cell floor(X0 - 0.5)
    // filaments (SGFD wall solid): node lists, first entry, count, (ds, Eh, EI)
    int n_fil, max_fil;
    const int32_t *fil_nodes, *fil_start, *fil_count;
    const double *fil_par;
};

// variants {min resident 256-thread blocks per SM, cells per thread}:
// 0 {6, 1} (40 registers), 1 {8, 1} (32), 2 {5, 1} (48), 3 {4, 2}, 4 {3, 2}
constexpr int SC_VARIANTS = 5;
int stream_collide_min_blocks(int variant);
int stream_collide_cells_per_thread(int variant);
// stream-collide of the stored cells [c0, c1) (c1 < 0: all cells); bump: the
// launch advances the step counter (one launch per step does)
cudaError_t launch_stream_collide(int prec, const void *fin, void *fout, const KParams &p, int block,
                                  int variant, cudaStream_t s, int desc = 0, int c0 = 0, int c1 = -1, int bump = 1);
cudaError_t launch_boundary(int prec, void *f, const KParams &p, const BcKParams &q, cudaStream_t s);
cudaError_t launch_gather(int prec, const void *fin, const KParams &p, int c0, int c1, double *f19, double *mac4,
                          cudaStream_t s);
cudaError_t launch_init_eq(int prec, void *fout, const KParams &p, const double *mac, int c0, int c1,
                           cudaStream_t s);
cudaError_t launch_wall_shear(int prec, const void *fin, const KParams &p, int c0, int c1, double *out3,
                              cudaStream_t s);
cudaError_t launch_state_rows(const BcState *st, const BcParam *par, const double *etab, int b0, int nb,
                              int nbc_total, long long steps, double *out8, cudaStream_t s);
cudaError_t launch_copy_words(const void *src, void *dst, size_t bytes, cudaStream_t s);
// per-step 0D input and output of lbm_step_io (see k_io_params, k_io_state)
cudaError_t launch_io_params(const double *params, int np, BcParam *par, const long long *cursor, cudaStream_t s);
cudaError_t launch_io_state(const BcState *st, const BcParam *par, const double *etab, int b0, int nb, int nbc_total,
                            const long long *step, double *out8, long long *cursor, cudaStream_t s);
cudaError_t launch_scatter_box(const double *mac4, int M, const int32_t *box, float *P, float *jx, float *jy,
                               float *jz, cudaStream_t s);
cudaError_t launch_cycle_change(const BcKParams &q, const int *bc_first, const int *n_bc, const long long *period,
                                long long steps, double *delta, int n_inst, cudaStream_t s);
cudaError_t launch_init(int prec, void *fout, const KParams &p, const double *f19, int c0, int c1,
                        cudaStream_t s);
// band velocities (unless band = false: issued earlier), node kernel, filaments
cudaError_t launch_ib(int prec, const void *fin, const KParams &p, const IbKParams &ib, cudaStream_t s,
                      bool band = true);
// the band-velocity pass over band-list entries [t0, t1), the node kernel over ib.order[k0 .. k1)
cudaError_t launch_band_moments(int prec, const void *fin, const KParams &p, const IbKParams &ib, int t0, int t1,
                                cudaStream_t s);
cudaError_t launch_ib_nodes(int prec, const KParams &p, const IbKParams &ib, int k0, int k1, cudaStream_t s);
cudaError_t prepare_filament_kernel(int max_fil);

}  // namespace lbm
