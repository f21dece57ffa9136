// lclb_internal.h -- host-side interface between the C ABI (lclb_api.cu) and
// the kernel launchers (lclb_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include "lclb_dev.cuh"

namespace lclb {

// mode bits
constexpr int FORCE_ACC = 1;  // accumulate colloid LC force/torque
constexpr int FORCE_FE = 2;   // write free-energy partials (one double per tile)
constexpr int LB_MOM = 1;     // write mass/momentum partials (4 doubles per tile)
constexpr int LC_RESID = 1;   // write residual partials (sum of squares, max; 2 doubles per tile)

// boundary links per link-exchange work unit
constexpr int LINK_CHUNK = 256;

// One work item of the persistent step kernel k_step: a tile (32 x ty x zc)
// of one phase of one box, a chunk of a box's boundary links, or a box's
// colloid update.  Before it runs, every counter wc[k] >= 0 must have
// reached wt[k]; when it is done, the counters dc[0], dc[1] (>= 0) are
// incremented.  part: index of the tile's residual partials (LC items).
enum { ITEM_STRESS = 0, ITEM_LB = 1, ITEM_LC = 2, ITEM_LINKS = 3, ITEM_COLLOID = 4 };
struct StepItem {
  int kind, box, x0, y0, z0, part;
  int wc[4], wt[4];
  int dc[2];
};

// export selectors (same values as LC_* in lc_lb.h)
constexpr int EXP_Q = 0, EXP_U = 1, EXP_RHO = 2, EXP_F = 3, EXP_FORCE = 4, EXP_SOLID = 5;

// One phase launch over a tile work list.
struct Launch {
  const DevBox* boxes;
  const int4* tiles;  // (box, x0, y0, z0)
  int ntiles;
  int zc;             // tile depth in z
  int ty;             // tile height in y (tile width in x is 32)
  int grid;           // blocks (persistent: tiles are strided over blocks)
  cudaStream_t stream;
};

cudaError_t launch_force(int prec, const Launch& L, int mode, double* part);
cudaError_t launch_lb(int prec, const Launch& L, int mode, double* part);
cudaError_t launch_flb(int prec, const Launch& L, int mode, double* part);  // ty in {4, 6, 8}
cudaError_t launch_lc(int prec, const Launch& L, int mode, double* part);
cudaError_t launch_stress(int prec, const Launch& L, int mode, double* part);  // H, P stored; colloid LC force
cudaError_t launch_lbp(int prec, const Launch& L, int mode, double* part);     // LB with the force from stored P
cudaError_t launch_links(int prec, const DevBox* boxes, const int2* chunks, int nchunks, int grid, cudaStream_t s);
cudaError_t launch_colloid(DevBox* boxes, int nboxes, cudaStream_t s);
// One coupled step (stress, LB, Q update, link exchange, colloid update of
// every box) as one persistent launch over the item list; sync holds the
// item counter (sync[0]) and the completion counters, zeroed before each
// launch.  commit = 0 leaves the state as it was (the colloid items only
// clear their sums): a timing run.  A wait that exceeds spin_limit polls
// sets *err and the item is skipped.
cudaError_t launch_step(int prec, int ty, DevBox* boxes, const StepItem* items, int nitems, int zc, unsigned* sync,
                        double* part, int spin_limit, int commit, int* err, int grid, cudaStream_t s);
int step_blocks_per_sm(int prec, int ty);
// Re-discretisation after the colloid update; mob lists (box, colloid) of mobile colloids.
cudaError_t launch_rediscretise(int prec, DevBox* boxes, int nboxes, const int2* mob, int nmob, int nsm,
                                cudaStream_t s);
cudaError_t launch_geometry(DevBox* boxes, int b, int N, cudaStream_t s);
cudaError_t launch_link_build(DevBox* boxes, int b, int N, int c, int* blocksum, int base, int* total,
                              cudaStream_t s);
cudaError_t launch_init_q(int prec, DevBox* boxes, int b, int N, int kind, const double* n, double amp,
                          unsigned long long seed, cudaStream_t s);
cudaError_t launch_set_field(int prec, DevBox* boxes, int b, int N, int which, const double* src, cudaStream_t s);
cudaError_t launch_export(int prec, const DevBox* boxes, int b, int N, int which, double* out, cudaStream_t s);
int diag_state_blocks(int N);
cudaError_t launch_diag_state(int prec, const DevBox* boxes, int b, int N, double* part, cudaStream_t s);
cudaError_t launch_reduce(const double* part, int rec0, int n, int w, unsigned maxmask, double* out, cudaStream_t s);

// Defect analytics of box b (lclb_defects.cu).  Labelling: parent[i] = the
// smallest node index of i's component of defect nodes, or -1; comp[root] =
// the component's rank in root order, list[rank] = root; blockcnt holds
// defect_blocks(N) ints; *total = number of components; *err set when a
// bounded loop gave up.  Statistics: size (ncomp ints), circ (6 ncomp),
// cen (3 ncomp), gyr (6 ncomp) doubles, size/circ/gyr zeroed by the caller.
int defect_blocks(int N);
cudaError_t launch_defects_label(int prec, const DevBox* boxes, int b, int N, double thr, int* parent, int* comp,
                                 int* list, int* blockcnt, int* total, int* err, cudaStream_t s);
cudaError_t launch_defects_stats(const DevBox* boxes, int b, int N, int ncomp, const int* parent, const int* comp,
                                 int* size, double* circ, double* cen, double* gyr, cudaStream_t s);

}  // namespace lclb
