// Device rebuild of the immersed-boundary structures after the Lagrangian
// points move (a moving or deforming wall): support origins, support slots and
// free masks on the finest level (Eq. 17), the A_F pattern (points whose 4x4x4
// supports overlap, Eq. 22) and the node -> (point, support index) spreading
// lists (Eq. 19).  Every list is sorted, so the sums over it run in the same
// order as after a host build.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ibg {

// Exclusive scan of n int32 values: out[0..n] (out[n] = total).  scratch holds
// scan_scratch_len(n) values.
int64_t scan_scratch_len(int64_t n);
void scan_excl(const int32_t* in, int32_t* out, int64_t n, int32_t* scratch, cudaStream_t st);

// error word codes of mv_supports
enum : int32_t { MV_OK = 0, MV_COARSE = 1, MV_NOFREE = 2, MV_OUTSIDE = 3 };

// The finest level's dense brick map and extents of one problem.
struct MoveGrid {
  const int32_t* bmap;     // [nb2][nb1][nb0] global brick of a level-L brick position, -1 absent
  int32_t nb[3];
  int64_t nf[3];           // finest cells per axis (nodes 0..nf)
  const uint16_t* meta;
  const double* origin;    // [3]
  const double* hf;        // [3]
  // coarse cells [n2][n1][n0]: refinement level of an active cell, 255 inactive;
  // a support node without a finest-level slot that is a vertex of an active
  // coarser cell exists on a coarser level (an error, as at setup)
  const uint8_t* cell_level;
  int32_t n[3];
  int32_t L;
};

// Support origins, slots and free masks of points 0..M-1; *err gets the
// largest error code met (MV_OK when every point is valid).
void mv_supports(const MoveGrid& G, int64_t M, const double* X, int32_t* org, int32_t* slot, uint64_t* freeb,
                 int32_t* err, cudaStream_t st);

// A_F pattern, pass 1: bins of 4 finest cells, per-row counts (rows M..Mt-1
// empty), rowptr = scan of the counts.  bins holds 3 * (nbins + 1) + M values.
int64_t mv_nbins(const MoveGrid& G);
void mv_af_count(const MoveGrid& G, int64_t M, int64_t Mt, const int32_t* org, int32_t* bins, int32_t* rcnt,
                 int32_t* rowptr, int32_t* scratch, cudaStream_t st);
// pass 2: columns of every row, sorted
void mv_af_fill(const MoveGrid& G, int64_t M, const int32_t* org, const int32_t* bins, const int32_t* rowptr,
                int32_t* col, cudaStream_t st);

// Spreading lists over ns slots: cnt, start, fill, flag, idx hold ns + 1
// values each; ent receives the entries (i * 64 + a) grouped by slot, sorted;
// sp_slot / sp_off the compact list of slots with entries.
void mv_spread(int64_t M, int64_t ns, const int32_t* slot, const uint64_t* freeb, int32_t* cnt, int32_t* start,
               int32_t* fill, int32_t* flag, int32_t* idx, int32_t* ent, int32_t* sp_slot, int32_t* sp_off,
               int32_t* scratch, cudaStream_t st);

}  // namespace ibg
