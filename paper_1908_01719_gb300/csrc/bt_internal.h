// Internal declarations of libbtgpu (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bt.h"

namespace bt {

// ---------------------------------------------------------------- host mesh
struct HostMesh {
  // input (copied)
  int64_t n_nodes = 0, n_tets = 0;   // elements: tetrahedra (nv = 4), triangles (3) or segments (2)
  int32_t n_cmpt = 0;
  int nv = 4;                          // nodes per element; faces have nv - 1 nodes
  bool surface = false;                // triangles of a surface in 3-D, not of the xy plane
  std::vector<double> xyz;          // 3 n_nodes
  std::vector<int32_t> tets;        // nv n_tets
  std::vector<int32_t> tet_cmpt;    // n_tets
  std::vector<double> D, kappa;     // n_cmpt
  uint32_t pmask = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  // derived on the host
  std::vector<int32_t> master;      // n_nodes -> master node
  std::vector<int32_t> tet_dof;     // nv n_tets
  std::vector<int32_t> dof_node, dof_cmpt;
  int64_t n_dof = 0;
  // interface faces (edges in 2-D): element a / element b, local vertex ids of
  // the face in element a, the 2 (nv - 1) dofs (side a, then the matching ones
  // of side b), kappa
  std::vector<int32_t> face_ta, face_tb;
  std::vector<int8_t> face_lv;      // (nv - 1) nf
  std::vector<int32_t> face_dof;    // 2 (nv - 1) nf
  std::vector<double> face_kappa;
  int64_t n_face = 0;
  // CSR pattern shared by every matrix
  std::vector<int64_t> row_ptr;     // n_dof + 1
  std::vector<int32_t> col;         // nnz
  int64_t nnz = 0;
  // slot-sorted element contributions: element entries (t nv^2 + i nv + j) and
  // face entries (f (2 fs)^2 + a 2 fs + b, fs = nv - 1), each in increasing
  // element order per slot
  std::vector<int64_t> tc_ptr, fc_ptr;  // nnz + 1
  std::vector<int32_t> tc, fc;
};

// Validates and builds everything above; returns BT_OK or BT_EINVAL with msg.
int build_host_mesh(HostMesh& m, std::string& msg);


// Halo tiles for the shared-memory SpMM: rows of each segment in Morton order
// of their node coordinates, cut greedily into tiles of at most `tmax` rows
// and `emax` entries whose columns span at most `umax` distinct rows of X
// (the tile's halo).
struct HaloTiles {
  int umax = 0;
  bool too_wide = false;          // some row has more than umax columns
  std::vector<int32_t> r0;        // [ntiles + 1] offsets into rows
  std::vector<int32_t> rows;      // [n] owned rows, tile by tile
  std::vector<int32_t> rowe;      // [n + 1] first entry of each owned row
  std::vector<int32_t> e0;        // [ntiles + 1] first entry of each tile
  std::vector<uint16_t> rowl;     // [n] local index of each owned row in its halo
  std::vector<int32_t> u0;        // [ntiles + 1] offsets into ucol
  std::vector<uint32_t> ucol;     // halo rows, ascending; bit 31: owned by the tile
  std::vector<uint16_t> lidx;     // [nnz] local column index of each entry
  std::vector<int32_t> slot;      // [nnz] CSR slot of each entry
  std::vector<int32_t> seg_tile0; // [G + 1]
};
void build_halo_tiles(const HostMesh& m, const std::vector<int64_t>& seg_row0, int umax, int tmax, int emax,
                      HaloTiles& t, bool sort_by_len = false);
// tile limits of the halo kernels: rows and entries per tile, and the shared
// memory (bytes) one block of the halo apply may use for its staged rows and
// entries
constexpr int HALO_TMAX = 128;
constexpr int HALO_EMAX = 448;
constexpr int HALO_SMEM_BUDGET = 96 * 1024;
// Configurations of the slice-tiled apply: the tile class (tile limits: halo
// rows, one 256-byte slice each in shared memory; owned rows; entries), the
// shared-memory stages of a block, its threads, the resident blocks per SM,
// and whether one warp of the block only copies (ws = 1: a producer warp fills
// the stages, the other warps take rows of the filled stages as they come,
// with per-stage mbarriers instead of block-wide barriers).  Configurations
// 0, 1 and 4 use the large tiles (class 0), 2 and 3 the small ones (class 1);
// the autotuner times all five.
struct SliceConf {
  int cls, umax, tmax, emax, stages, threads, blocks, ws;
};
constexpr int SLICE_NCONF = 5, SLICE_NCLS = 2;
constexpr SliceConf SLICE_CONF[SLICE_NCONF] = {{0, 256, 128, 1536, 2, 512, 1, 0},
                                               {0, 256, 128, 1536, 1, 256, 2, 0},
                                               {1, 128, 64, 1024, 2, 256, 2, 0},
                                               {1, 128, 64, 1024, 1, 256, 3, 0},
                                               {0, 256, 128, 1536, 2, 512, 1, 1}};

// Weak pseudo-periodic coupling of the box faces (artificial permeability,
// Appendix B): the boundary-face mass B on both sides of every selected axis
// (as values on the CSR slots) and the face-mass coupling of each face with
// its partner face, as rows of (col, weight, axis | sign << 2) sorted by row.
// The mesh must match across the box (partner node at x + L_k e_k).
struct WeakPeriodic {
  std::vector<double> B;        // [nnz] boundary-face mass per slot
  std::vector<int32_t> rows;    // [nr] boundary dofs with coupling entries
  std::vector<int32_t> ptr;     // [nr + 1]
  std::vector<int32_t> col;     // partner dof
  std::vector<double> w;        // face-mass weight
  std::vector<int8_t> code;     // axis (bits 0-1), sign bit 2 (set = -1)
  double L[3] = {0, 0, 0};      // box lengths
  double h = 0;                 // (6 x mean tetrahedron volume)^(1/3)
};
int build_weak_periodic(const HostMesh& m, uint32_t axes, WeakPeriodic& wp, std::string& msg);

// ---------------------------------------------------------------- device helpers
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    free();
    n = count;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)&p, count * sizeof(T));
  }
  void free() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~DBuf() { free(); }
};

// Step coefficients of the generic operator
//   y_r = a * (P0 x_r) + bq2 * q_r^2 * (P1 x_r) + i * cq * q_r * (sum_k qhat_k P_{2+k}) x_r
// where P0 is A0 or K+J, P1 the D-weighted mass (transformed frame only) and
// P2..P4 the direction planes (Mx,My,Mz in the lab frame, Ex,Ey,Ez in the
// transformed frame).
struct OpCoef {
  double a;
  double bq2;
  double cq;
};

// Double-float plane: value = hi + lo, both FP32.
struct DFPlanes {
  float* hi = nullptr;
  float* lo = nullptr;
};

}  // namespace bt
