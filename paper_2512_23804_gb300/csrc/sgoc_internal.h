// Internal definitions of the SG optimal-control solver library.
#pragma once

#include <cmath>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sgoc.h"

namespace sgoc {

// Thread-local message for sgoc_last_error().
void set_error(const std::string& msg);

#define SGOC_CUDA_TRY(expr)                                                       \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ::sgoc::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));      \
      return SGOC_ERR_CUDA;                                                       \
    }                                                                             \
  } while (0)

#define SGOC_TRY(expr)                      \
  do {                                      \
    sgoc_status s_ = (expr);                \
    if (s_ != SGOC_OK) return s_;           \
  } while (0)

// E[xi psi_n psi_{n+1}] for orthonormal Legendre polynomials psi_n = sqrt(2n+1) P_n,
// xi ~ U[-1,1], from the three-term recurrence xi P_n = ((n+1) P_{n+1} + n P_{n-1})/(2n+1).
inline double legendre_coupling(int n) {
  return (n + 1) / std::sqrt((2.0 * n + 1.0) * (2.0 * n + 3.0));
}

// One level of the geometric hierarchy for the mean operator: a constant
// 9-point stencil (centre, edge, corner) on an nx-element grid.
struct Level {
  int nx;        // elements per side
  int n1;        // interior nodes per side = nx - 1
  int64_t n;     // n1 * n1
  double diag, edge, corner;
};

// Slot table of one SG launch shape (output columns [out0, out1), input columns
// [in0, in1), couplings k < kmax) for the two-phase SG kernel: every input
// column alpha gets one slot per KL index k its outputs use (bit k of mask,
// slots numbered from base in increasing k); every output column beta gets the
// slot of (beta, 0) and a list of (slot, coefficient) pairs in table order.
struct UTab {
  int in0 = 0, in1 = 0, out0 = 0, out1 = 0, kmax = 0;
  int nslots = 0, nent = 0;
  std::vector<int> mb;        // 2 per input column: mask, base
  std::vector<int> diag;      // per output column
  std::vector<int> eptr;      // per output column + 1
  std::vector<int> eslot;     // per entry
  std::vector<double> ec;     // per entry
  int* d_mb = nullptr; int* d_diag = nullptr; int* d_eptr = nullptr;
  int2* d_e32 = nullptr;      // (32 * slot, float bits of c) per entry
  int* d_eslot = nullptr; double* d_ec64 = nullptr;
};

// Device pointers into the caller's persistent buffer.
struct DevData {
  double* kap64 = nullptr;     // (M+1) x nx x nx, kappa_k(e) / 6
  float* kap32 = nullptr;
  int* nbr_ptr = nullptr;      // CSR over output columns beta: P + 1
  int* nbr_end_r = nullptr;    // per column: end of the entries with k < r (truncation)
  int* nbr_end_all = nullptr;  // per column: end of all entries
  int* nbr_alpha = nullptr;    // neighbour column alpha = beta +- e_k
  int* nbr_k = nullptr;        // KL index k (1..M)
  double* nbr_c64 = nullptr;   // E[xi_k Psi_alpha Psi_beta]
  float* nbr_c32 = nullptr;
  int* dn_ptr = nullptr;       // downward part of the neighbour table (alpha one level below beta)
  int* dn_end_r = nullptr;
  int* dn_alpha = nullptr;
  int* dn_k = nullptr;
  double* dn_c64 = nullptr;
  float* dn_c32 = nullptr;
  // square-root-free Cholesky M1 = L D L^T of the 1-D mass matrix (h/6) tridiag(1, 4, 1):
  // subdiagonal l_i of L (l_0 = 0) and 1 / D_i, n1 entries each (the exact mass solve)
  double* mass_l64 = nullptr; double* mass_id64 = nullptr;
  float* mass_l32 = nullptr; float* mass_id32 = nullptr;
  void* spec_img = nullptr;    // exact mean solves: constant image of spectral_image(n1)
  double* yhat = nullptr;      // slabs x n target values
  double* y0 = nullptr;        // n initial state (zeros when absent)
};

}  // namespace sgoc

struct sgoc_problem {
  // problem statement
  int nx = 0, M = 0, p = 0, nt = 0;
  int chaos = 0;                     // 0 Legendre / affine, 1 Hermite / chaos-expanded coefficient
  int nterms = 1;                    // coefficient planes: M + 1, or C(M + 2p, 2p)
  int lev_dist = 1;                  // largest chaos-level distance of a kept coupling
  bool sgr_ok = false;               // the register SG kernel is compiled for this (M, p) in this index order
  bool spec = false;                 // the fast-diagonalisation image is uploaded (exact mean or mass solves)
  double length = 1.0;               // side of the square domain
  double beta = 0, gamma = 0, T = 1, tau = 1, kappa0 = 1, s = 0;  // s = sqrt((1+gamma)/beta)
  int n1 = 0, P = 0, slabs = 1;
  int64_t n = 0, F = 0, N = 0;       // F = slabs * P * n, N = 3F
  std::vector<double> kappa, yhat, y0;
  sgoc_options opt{};
  int r = 1;                         // truncation
  // chaos basis
  std::vector<int32_t> idx;          // P x M
  std::vector<int32_t> tidx;         // n_terms x M coefficient-term multi-indices (Hermite)
  std::vector<int> off;              // p + 2 level offsets
  std::vector<int> nbr_ptr, nbr_alpha, nbr_k, nbr_end_r;
  std::vector<double> nbr_c;
  std::vector<int> dn_ptr, dn_alpha, dn_k, dn_end_r;   // downward part (one level below)
  std::vector<double> dn_c;
  // multigrid hierarchy of the mean operator (level 0 = finest)
  std::vector<sgoc::Level> levels;
  double mass_h2_36 = 0;             // h^2 / 36 on the finest grid
  std::vector<double> dweights;      // time weights D_t (1 when steady)
  // SG launch shapes: [0] the full operator (all columns, all k), [1 + d] the hGS visit of level d,
  // [2 + p + d] the first (ascending) hGS visit of level d: couplings to level d - 1 only
  std::vector<sgoc::UTab> utabs;
  // device
  sgoc::DevData dev;
  bool uploaded = false;
  size_t persistent_bytes = 0;
  void* runtime = nullptr;           // host-side solve resources (solver.cu)
};

namespace sgoc {

// Workspace needs for one precision (bytes), see solver.cu.
size_t workspace_bytes(const sgoc_problem* pb, int precision);
size_t precond_workspace_bytes(const sgoc_problem* pb, int esize);
int level_columns_max(const sgoc_problem* pb);
void release_runtime(sgoc_problem* pb);
// Captured graphs refer to device addresses of the problem data: drop them on re-upload.
void invalidate_graphs(sgoc_problem* pb);

}  // namespace sgoc
