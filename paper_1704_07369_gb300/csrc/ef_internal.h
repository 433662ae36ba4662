// ef_internal.h -- structures shared by the host plan code (ef_plan.cpp) and the CUDA kernels.
#pragma once

#include <cstdint>

namespace ef {

// One step of the per-cell direction loop.  Each op runs the inverse transform of one spectral
// multiply M_dir(l) * Fhat(l) (Sec. 4.1, eq. fastAlg with the filter folded into M), or of two
// (dir, dir2) for the paired kinds, and folds the real-space results into the accumulators.
// Single-slab mode (one shared-memory slab, S and G accumulators):
//   OP_S_SET   S  = w a            OP_S_ADD  S += w a
//   OP_G_SET   G  = a S            OP_G_ADD  G += a S
//   OP_LOSS    nu = a;  Q = G - F nu   (the gain/loss split of Sec. 3.1.2, eq. def_A)
// Paired mode (two slabs, G only):
//   OP_NU_INIT     nu = a;  G = -F nu       (first op)
//   OP_PAIR        G += a b                 (a = dir, b = dir2)
//   OP_PAIR_LAST   Q = G + a b; output      (last op)
enum OpKind : int {
    OP_S_SET = 0, OP_S_ADD = 1, OP_G_SET = 2, OP_G_ADD = 3, OP_LOSS = 4, OP_NU_INIT = 5,
    OP_PAIR = 6, OP_PAIR_LAST = 7
};

struct Op {
    int dir;        // row of the multiplier table
    int kind;       // OpKind
    double w;       // weight (S ops)
    int dir2;       // second row (paired kinds)
    int pad;
};

enum OutMode : int { OUT_COLLIDE = 0, OUT_EULER = 1 };

constexpr int kMaxOps = 512;
constexpr int kDiag = 10;

// Kernel arguments for one size class (all cells of one N).
struct CollideArgs {
    const void *F;            // input cells (element type Tr)
    void *Q;                  // output cells (OUT_COLLIDE) or F itself (OUT_EULER, in place)
    const int64_t *cell_off;  // device: element offset of each cell of the class (null: c * N^d)
    const int64_t *cell_id;   // device: global cell index of each cell of the class (null: c)
    int64_t ncells;           // cells in this class
    const void *mult;         // device: multiplier tables [ndir][N1 * H][N]... see layout below
    const Op *ops;            // device: op list
    int nops;
    int cluster;              // CTAs per cell
    int planes;               // axis-0 planes per CTA = N / cluster
    int sg_global;            // 1: S and G accumulators in global workspace, 0: shared memory
    void *sg_ws;              // global S/G workspace (sg_global), [slot][2][planes*N1*(N+1)]
    int out_mode;             // OutMode
    double dt;                // Euler step
    double h;                 // grid spacing 2L/N
    double *diag;             // nullable: [cell_id][kDiag]
    int *status;              // device status word
    unsigned long long *counter;  // nullable: dynamic cell queue (zeroed before the launch)
    int prefetch;             // 1: prefetch the next op's multipliers into L1
    int paired;               // 1: two spectral slabs per CTA and the paired op kinds
    const long long *dev_ncells;  // nullable: cell count read from device memory at kernel start
    void *fh_ws;              // forward spectrum workspace: per cluster slot N * NP complex, [z][p]
    int npc;                  // axis-0 pencils per CTA (even; CTA r owns [r npc, (r + 1) npc) of NP)
};

// Arguments of the low-mode feature kernel (one launch per size class).
struct FeatArgs {
    const void *F;                           // cells of N^d values (element type of the plan), 16-byte aligned
    const int64_t *cell_off;                 // nullable: element offset of cell c (default c * N^d)
    const int64_t *cell_id;                  // nullable: output row of cell c (default c)
    int64_t ncells;                          // cells (upper bound when dev_ncells is set)
    const unsigned long long *dev_ncells;    // nullable: number of cells, read on the device
    int log_input;                           // field 0 is ln max(F, 1e-30) instead of F
    float *feat;                             // [row][fstride]: field 0, (re, im) per slot
    float *featL;                            // nullable: field 1 = modes of ln max(F, 1e-30)
    int fstride;
    double *mom;                             // nullable: [row][kDiag] moments of F (no Q entries)
    double h;                                // grid spacing 2L/N
    const int *modes;                        // device [nmodes][3]: (k_axis0, k_axis1, k_axis2); 2D: (0, k0, k1)
    int nmodes;
};

// Multiplier table layout for one class: mult[dir][lz][p], p = ly * H + lx (3D) or p = lx (2D),
// H = N/2 + 1, lz in [0, N) in FFT order; the loss table is the last dir.

}  // namespace ef
