// Internal declarations shared by the translation units of liblelbm: the device
// code (lelbm_step.cu, lelbm_cell.cu, lelbm_batch.cu, lelbm_noalloc.cu,
// lelbm_mlp.cu) and the C ABI (lelbm_api.cu, host side).
#pragma once

#include <type_traits>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lbm {

// Cell kinds of the padded grid.
enum : uint8_t { CELL_FLUID = 0, CELL_PAD_IN = 1, CELL_PAD_OUT = 2, CELL_SOLID = 3 };

// Arithmetic of the step (the values of LELBM_FP64, LELBM_MIXED, LELBM_FP32).
enum : int { PREC_FP64 = 0, PREC_MIXED = 1, PREC_FP32 = 2 };
// storage type of a cell's normalised constraints: the FP32 path computes them in FP32
template <int PREC>
using Con = typename std::conditional<PREC == PREC_FP32, float, double>::type;
// Threads per block of the cell update.  The mixed path runs one block of twelve warps per
// SM: its block-synchronous phases then hold every scheduler of the SM at the same code
// (one phase's instructions in the instruction caches at a time).
template <int PREC>
constexpr int cell_threads() { return PREC == PREC_MIXED ? 384 : 128; }

// Physical and numerical constants of one handle (Sec. II, App. C, App. D).
struct Model {
    double K;           // internal degrees of freedom
    double inv_dk;      // 1 / (D + K)
    double nu_s;        // kinematic shear viscosity
    double nu_b;        // kinematic bulk viscosity, < 0 -> omega_b = 1
    double Pr;          // Prandtl number
    int limiter;        // Knudsen limiter on
    double n_conf;      // conformation number n
    double r_min;       // minimum acoustic radius
    double refine_div;  // divisor in N_r
    double refine_rad;  // refinement radius factor
    int max_refine;     // cap on N_r (<= 4)
    double tol;         // EPR tolerance, thermal units
    int max_iter;       // Newton update cap
    float* rec_x;                  // record mode: per-cell features, or null
    float* rec_y;                  // record mode: per-cell targets, or null
    const __nv_bfloat16* mlp_w;    // learned warm start: BF16 weights, or null
    const float* mlp_nrm;          // learned warm start: normalisation
    float* lam_store;              // stored warm start: per-cell multiplier corrections, SoA
                                   // [NF + NG][ncell], or null
    const float* mlp_start;        // learned warm start of this step: per-cell corrections from
                                   // mlp_start_kernel, SoA [NF + NG][ncell] (NaN: none), or null
    float mlp_gate;                // learned start only where the normalised constraints depart
                                   // from equilibrium by at least this much (0: everywhere)
    double* det_lam;               // deterministic streaming (FP64 2D): the cell kernel writes
                                   // each cell's final multipliers here, SoA [NF + NG][ncell],
                                   // instead of scattering; null: scatter with atomics
    int* det_halo;                 // with det_lam: max over cells of the reach of the velocity
                                   // set (cells), for the gather's window
    // FP32 copies for the FP32 path (set by set_fp32_params)
    float K32, nu_s32, nu_b32, Pr32, n_conf32, r_min32, refine_div32;
    double rad2_32[5];  // squared refinement radii, FP32 arithmetic: (refine_rad / 2^L)^2
};

// Fills the FP32 copies of the model parameters (host).
inline void set_fp32_params(Model& m) {
    m.K32 = (float)m.K;
    m.nu_s32 = (float)m.nu_s;
    m.nu_b32 = (float)m.nu_b;
    m.Pr32 = (float)m.Pr;
    m.n_conf32 = (float)m.n_conf;
    m.r_min32 = (float)m.r_min;
    m.refine_div32 = (float)m.refine_div;
    float rad = (float)m.refine_rad;
    for (int L = 0; L < 5; L++) {
        const float r2 = rad * rad;
        m.rad2_32[L] = (double)r2;
        rad *= 0.5f;
    }
}

// Padded-grid geometry.  2D: one instance, cell = iy * NX + ix.
// 1D: n_inst instances concatenated, each [pad | n | pad] (no pads if periodic).
struct Geometry {
    int D;
    int NX, NY;
    long long ncell;
    int nx, ny, pad;
    int periodic[2];
    int n_inst;
    const int* inst_of_cell;     // 1D: instance of every cell
    const long long* inst_lo;    // 1D: first interior cell of each instance
    const int* inst_n;           // 1D: interior length of each instance
    const uint8_t* wall_dist;    // 2D with solids: Chebyshev distance (cells) from each
                                 // cell to the nearest solid cell, capped at 255; else null
    const uint8_t* noslip;       // 2D with no-slip walls: per solid cell 1 for a no-slip wall
                                 // at rest, 2 for one moving at wall_u (0: slip wall); null if none
    double wall_u[2];            // velocity u_w of the moving no-slip walls (Eq. IIIB2-IIIB4)
};

// Padded 3D grid: cell = (iz * NY + iy) * NX + ix; p* = pad layers of each axis (0 on a
// periodic axis).
struct Geometry3 {
    int NX, NY, NZ;
    long long ncell;
    int nx, ny, nz;
    int px, py, pz;
    int periodic[3];
};

// Device-side counters (all 64-bit, updated with atomics).
struct DevStats {
    unsigned long long cells;
    unsigned long long newton_hist[64];
    unsigned long long fallback_eq;
    unsigned long long fallback_mx;
    unsigned long long q_max;
    unsigned long long disp_max_bits;  // bit pattern of a non-negative double
    unsigned long long first_fail;     // smallest failing cell, ~0ull if none
    unsigned long long points_f;       // stencil points of fluon Newton passes
    unsigned long long points_g;       // stencil points of phonon Newton passes
    unsigned long long points_ms;      // stencil points streamed
    unsigned long long points_32;      // stencil points of FP32 Newton passes (mixed and FP32 paths)
    unsigned long long judge_redo;     // mixed path: cells whose FP64 check failed and were re-solved
    unsigned long long mlp_retry;      // cells whose learned start failed and were re-solved from Eq. IID13
    unsigned long long wall_hits;      // streamed populations reflected at a solid face (Sec. III.B)
    unsigned long long mlp_cells;      // cells given the learned warm start
    unsigned long long points_df;      // stencil points of double-float streaming passes (mixed path)
    unsigned long long points_df_corr; // stencil points of double-float correction passes (mixed path)
};

void launch_fill_pads(int D, const Model& m, const double inlet[4], double* M, long long ncell,
                      const long long* pad_cell, const long long* pad_src, long long npad,
                      cudaStream_t s);
void launch_cell_update(const Model& m, const Geometry& g, const uint8_t* type, const double* Min,
                        double* Mout, DevStats* st, unsigned long long* work, int grid_blocks, int prec,
                        cudaStream_t s);
void launch_eq_state(int D, double K, const uint8_t* type, const double* rho, const double* u,
                     const double* RT, double* M, long long ncell, cudaStream_t s);
void launch_macros(int D, double K, const uint8_t* type, const double* M, double* rho, double* u,
                   double* RT, long long ncell, cudaStream_t s);
int cell_update_blocks(int D, int prec, int device);
void launch_batch_persistent(const Model& m, const Geometry& g, const double inlet[4], int bc_left_inflow,
                             int bc_right_inflow, const uint8_t* type, double* A, double* B, DevStats* st,
                             unsigned long long* work, const int* order, const long long* inst_first,
                             const int* inst_pad, int* steps_left, int nsteps, int blocks, int threads, int prec,
                             cudaStream_t s);
int batch_persistent_max_blocks_per_sm(int prec, int threads);
double fma_peak(int fp64, int device);
void launch_mlp_infer(int D, const __nv_bfloat16* W, const float* nrm, const float* X, long long n, float* Y,
                      cudaStream_t s);
void launch_mlp_start(const Model& m, const Geometry& g, const uint8_t* type, const double* Min, float* out,
                      int device, cudaStream_t s);

// 3D (lelbm_3d.cu): inlet = (rho, ux, uy, uz, RT).
void launch_fill_pads3(const Model& m, const double inlet[5], double* M, long long ncell, const long long* pad_cell,
                       const long long* pad_src, long long npad, cudaStream_t s);
void launch_cell3d(const Model& m, const Geometry3& g, const double* Min, double* Mout, DevStats* st,
                   unsigned long long* work, int blocks, cudaStream_t s);
int cell3d_blocks(int device);
// Deterministic moment streaming (lelbm_gather.cu): every target cell of a padded 2D grid
// sums, in a fixed order, what the cells within reach send it, from the multipliers the
// FP64 cell kernel left in m.det_lam.
void launch_gather2d(const Model& m, const Geometry& g, const double* Min, double* Mout, DevStats* st,
                     cudaStream_t s);

// One object file per kernel variant (lelbm_cell.cu, lelbm_batch.cu).
template <int D, int PREC>
struct CellVariant {
    static void launch(const Model& m, const Geometry& g, const uint8_t* type, const double* Min, double* Mout,
                       DevStats* st, unsigned long long* work, int blocks, size_t smem, cudaStream_t s);
    static int blocks_per_sm();
};

template <int PREC>
struct BatchVariant {
    static void launch(const Model& m, const Geometry& g, const double inlet[4], int bc_left_inflow,
                       int bc_right_inflow, const uint8_t* type, double* A, double* B, DevStats* st,
                       unsigned long long* work, const int* order, const long long* inst_first, const int* inst_pad,
                       int* steps_left, int nsteps, int blocks, int threads, size_t smem, cudaStream_t s);
    static int blocks_per_sm(int threads);
};

}  // namespace lbm
