// Kernel argument blocks and launcher declarations shared by the library's
// translation units (host API, step kernel, inlet kernel).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace stg {

// Step counter on the device.  Step t reads t[t & 1]; the fused step kernel
// writes t[(t + 1) & 1] = t + 1 when it finishes, so a captured graph can be
// replayed without host-side parameter updates.
struct StepCtl {
    long long t[2];
    long long t0_filter;  // step at which the temporal filter restarts
    unsigned long long err; // error bits set by kernels (none of the current kernels sets one)
};

struct StepArgs {
    const void *src;      // post-collision populations of the previous step
    void *dst;            // post-collision populations of this step
    // per-population plane pointers (kernel parameters, so every address is
    // one multiply-add of the cell index onto a constant-bank operand):
    //   srcp[i] = plane i of src, srci[i] = srcp[i] - (c_ix + c_iy nx) elements
    //   (interior pull), dstp[i] = plane i of dst
    //   srcy[i] = srcp[i] - c_iy nx elements (two-cells-per-thread pull)
    const void *srcp[19];
    const void *srci[19];
    const void *srcy[19];
    void *dstp[19];
    int il, ir;             // 32-wide x chunks [il, ir) of rows 1..ny-2 belong to the interior kernel
    int interior;           // interior kernel: 0 best available, 1 one cell per thread, 2 cell pairs
    int aa;                 // 1: one lattice updated in place (AA pattern; src == dst), 0: two lattices
    // tile of the plain (non-sampling) vector launches: layout 0 = 8 z-warps on one 64-cell x chunk,
    // layout 1 = 4 x-warps (256 cells) walking z together; zc / wall_zc = z planes per block of the
    // rows 1..ny-2 / wall-row launch (0: the whole z column)
    int tile_layout, tile_zc, tile_wall_zc;
    unsigned total_blocks;  // blocks of all step kernels of the pass (mass-check completion count)
    int slot_base;          // first mass-partial slot of this launch's blocks
    int bump_t;             // this launch advances the device step counter
    int nx, ny, nz;
    unsigned P;           // cells per population plane (nx*ny*nz)
    int bc_x, bc_y;       // STG_BC_X_*, STG_BC_Y_*
    float tau0, kq;       // kq = 18 sqrt(2) C  (eq. tau_eff)
    float Fx, Fy, Fz;
    int has_force;
    const float *ubc;     // inlet velocity plane [3][nz][ny]
    const float *spf;     // sponge zone: viscosity factor per column x [nx] (eq. sponge_visco); nullptr: off
    StepCtl *ctl;
    int parity;
    int stats_every, check_every;
    double *stat_mean;    // [3][ny][nx]
    double *stat_rey;     // [6][ny][nx]
    float *stat_part;     // sampling steps of the vector kernels: FP32 sums per group of
                          // STAT_GROUP z planes, [ceil(nz / STAT_GROUP)][9][ny][nx]
    double *mass_partial; // [gridDim.x * gridDim.y]
    unsigned *mass_counter;
    double *mass_out;     // [0]: last checked mass
};

struct InletArgs {
    int ny, nz, N;
    const float *A;       // [N][ny]  k^n d^n_y (j + 1/2) mod 2 pi
    const float *B;       // [N][nz]  k^n d^n_z k       mod 2 pi
    const float *SQ;      // [N][ny]  sqrt(6 q^n(y_j))
    const float *sig;     // [N][3]   sigma^n
    const unsigned long long *phq;  // [N] phi^n / (2 pi) as a Q0.64 fraction of a turn
    const unsigned long long *omq;  // [N] phase advance per step, -d^n_x U_b / max l_e turns, Q0.64
    const float *a6;      // [ny][6]  Cholesky factor a11 a21 a22 a31 a32 a33
    const float *u_int;   // [ny]     interpolated mean streamwise velocity
    float a_filter;
    float *uf;            // [3][nz][ny] filtered fluctuation (state)
    float *ubc;           // [3][nz][ny] inlet velocity output
    int ahead;            // the plane is for step t + ahead (t = ctl->t[parity])
    StepCtl *ctl;
    int parity;
};

struct MassArgs {
    const void *src;
    unsigned P;
    int storage;
    double *partial;
    unsigned *counter;
    double *out;
};

// launchers (return the launch status)
// `stats` must be true exactly on sampling steps ((t + 1) % stats_every == 0);
// the host tracks t and decides.
// inlet: the inlet kernel for the next step's plane (NULL: none), launched on the branch
cudaError_t launch_step(const StepArgs &a, int storage, int collision, bool stats,
                        cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join,
                        const InletArgs *inlet = nullptr);
// binary16 regularized unforced lattices take quads (four cells per lane)
// when the rows split into whole quads
inline bool quads_fit(int nx) { return nx % 4 == 0 && nx >= 8; }
cudaError_t launch_inlet(const InletArgs &a, cudaStream_t s);
// FP64 Cholesky factor of the lattice-unit Reynolds stress per inlet node (setup)
cudaError_t launch_setup_nodes(int ny, const double *R6, float *a6, cudaStream_t s);
// swap: store population i in slot opp(i) (the in-place layout before a step of even index)
cudaError_t launch_init_equilibrium(void *dst, int storage, int nx, int ny, int nz, const float *u_int, int swap,
                                    cudaStream_t s);
cudaError_t launch_mass(const MassArgs &a, cudaStream_t s);
// How to find a population in a stored lattice: slot i of the cell for two
// lattices, the in-place arrangement after t completed steps otherwise.
struct LatticeView {
    int nx, ny, nz, bc_x, bc_y, aa;
    size_t P;
    long long t;
};
// velocity of n cells (xyz: device int triples) of a stored lattice into out[3 n]
cudaError_t launch_probe(const void *src, int storage, const LatticeView &lv, int n, const int *xyz, float Fx,
                         float Fy, float Fz, float *out, cudaStream_t s);
// canonical sub-block [19][bz][by][bx] of a stored lattice into device memory `out`
cudaError_t launch_gather_block(const void *src, int storage, const LatticeView &lv, int x0, int y0, int z0, int bx,
                                int by, int bz, void *out, cudaStream_t s);

// Upper bound of the mass-partial slots of one step pass over every tile
// that set_tile accepts (z chunks of at least MIN_ZC planes).
constexpr int MIN_ZC = 4;
// z planes per block on sampling steps of the vector kernels (fixed, so the
// statistics do not depend on the launch tile)
constexpr int STAT_GROUP = 32;
int step_grid_blocks(int nx, int ny, int nz);
int mass_grid_blocks();

}  // namespace stg
