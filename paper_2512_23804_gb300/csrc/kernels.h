// Launchers of the device kernels (templated on the vector type T = float or double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sgoc {

// Number of kernels this library has launched in the process (all streams).
int64_t kernel_launches();
// The next kernel this library launches on `st` takes a full stream dependency
// (no programmatic overlap): call after a cross-stream event wait, a copy or a
// graph launch on `st`.
void pdl_fence(cudaStream_t st);
// Whether the next launch on `st` must take the full dependency (and clear the mark).
bool pdl_take_fence(cudaStream_t st);
void add_launches(int64_t n);
bool profile_enabled();

// Optional per-kernel-class timing: when enabled, every launch is bracketed by
// CUDA events on its stream and its algorithmic bytes/flops are recorded.
enum KernelKind {
  KK_SG = 0, KK_MASS, KK_CHEB, KK_SMOOTH, KK_RESIDUAL, KK_RESTRICT, KK_PROLONG, KK_VCYCLE_FUSED,
  KK_DOT, KK_SCALAR, KK_VECTOR, KK_MEAN_EXACT, KK_COUNT
};
const char* kernel_kind_name(int kind);
void profile_enable(bool on);
bool profile_query(int kind, int64_t* launches, double* ms, double* bytes, double* flops);
struct ProfScope {
  ProfScope(int kind, cudaStream_t st, double bytes, double flops);
  ~ProfScope();
  int kind; cudaStream_t st; int slot;
};

// out[t][beta] = cr*R + c0*(K_0 X)[beta] + c1*sum_{k=1}^{kmax-1} (K_k X G_k)[beta]
//              + cm*(M X)[beta] + cy*out_old,   beta in [out0, out1), t < nslabs.
// X is read in columns [in0, in1) (must contain every neighbour of the output
// columns and the output columns themselves).  Column beta of slab t of an
// operand Z lives at Z + t*zs + (beta - zcol0)*n.
template <typename T>
struct SGArgs {
  const T* X; int64_t xs;
  T* Y; int64_t ys; int ycol0;
  const T* R; int64_t rs; int rcol0;
  int n1; int64_t n; int nx; int M;
  int out0, out1, in0, in1, kmax, nslabs;
  T c0, c1, cm, cr, cy;
  T mass;                       // h^2/36
  const T* kap;                 // kappa_k(e)/6, (M+1) x nx x nx
  const int* nbr_ptr; const int* nbr_alpha; const int* nbr_k; const T* nbr_c;
  const int* nbr_end;           // per output column: end of its entries with k < kmax
  double deg_sum;               // number of (beta, neighbour) pairs used (work accounting only)
  int nnz_out;                  // neighbour-table entries of the output columns (all k)
  // slot table of this launch shape (two-phase kernel; null: the one-phase kernels)
  const int* u_mb; const int* u_diag; const int* u_eptr; const int2* u_e32;
  int u_nslots, u_nent;
  // 1: the outputs' own columns take no part (no kappa_0 or mass term, c0 and cm unused);
  // the output range then need not lie inside the input range
  int no_own;
  // Legendre chaos of total degree p (the register kernel, variant 7, is compiled for a few
  // (M, p)); -1 otherwise.  cup[j] = E[xi psi_j psi_(j+1)], the couplings of G_k by the k-th
  // component j of the lower multi-index (equal to the table's float values).
  int legendre_p = -1;
  T cup[11];
};
template <typename T>
cudaError_t launch_sg(const SGArgs<T>& a, cudaStream_t st);
// Merged launches over several problems of one launch shape (same grid, chaos levels,
// truncation, slabs and epilogue terms): member g's operands, coefficient data and
// scalars replace those of the shared SGArgs in the CTAs of slabs [g*nslabs, (g+1)*nslabs)
// of grid dimension z.  Member 0 is the SGArgs itself.  Every member's outputs are
// computed exactly as by a launch of its own.
constexpr int kMaxGroup = 8;
template <typename T>
struct SGMulti {
  int ng = 1;
  const T* X[kMaxGroup]; T* Y[kMaxGroup]; const T* R[kMaxGroup]; const T* kap[kMaxGroup];
  T c0[kMaxGroup], c1[kMaxGroup], cm[kMaxGroup], cr[kMaxGroup];
};
template <typename T>
cudaError_t launch_sg_group(const SGArgs<T>* a, int ng, cudaStream_t st);
// SG kernel variants (0 one-phase, 1 quad 32-node tile, 2 quad 16-node tile,
// 3 two-phase float32, 4 and 5 the quad tiles at four CTAs per SM, 6 direct:
// a thread per node and output, feasible while outputs + couplings <=
// kSGDirectMaxTerms; 7 register form: float32 Legendre chaos of a compiled (M, p),
// a thread per node with every output column's sum in registers) and the
// process-wide tuning cache keyed by launch shape.  Variants 0-6 agree bit for bit;
// 7 sums a column's coupling terms in another order and agrees with them to rounding.
constexpr int kSGVariants = 8;
// The multi-indices (count x M, row-major) the register SG kernel was compiled with for
// (M, p); false when it is not compiled for them.
bool sgr_indices(int M, int p, std::vector<int>& out);
constexpr double kSGDirectMaxTerms = 256;
template <typename T>
cudaError_t launch_sg_variant(const SGArgs<T>& a, int variant, cudaStream_t st,
                              const SGMulti<T>* mg = nullptr);
template <typename T>
bool sg_variant_feasible(const SGArgs<T>& a, int variant);
template <typename T>
int sg_tuned_variant(const SGArgs<T>& a);          // -1: not tuned
template <typename T>
void sg_set_variant(const SGArgs<T>& a, int variant);
template <typename T>
void sg_clear_variant(const SGArgs<T>& a);
void sg_clear_tuning();

// out[t][c] = cy*out_old + sum_j a_j w_j(c,t) (M V_j[t + shift_j])[c] + ar*R[t][c]
// for columns c in [0, ncols) of each slab (column c is global column col0 + c).
// Weight flags: bit 0 multiplies by H^gamma(col) = (col == 0 ? 1 : 1 + gamma),
// bit 1 by D_t (1/2 at the first and last of nt >= 2 steps, else 1).
template <typename T>
struct MassArgs {
  T* out; int64_t os;
  int ncols, col0, nslabs, n1; int64_t n;
  T mass, cy, ar, gamma;
  int nt;
  int nv;
  const T* V[3]; int64_t vs[3]; int shift[3]; T a[3]; int wflags[3];
  const T* R; int64_t rs;
};
template <typename T>
cudaError_t launch_mass(const MassArgs<T>& a, cudaStream_t st);

// Chebyshev semi-iteration for M X = B on ncols columns of n entries
// (textbook Golub-Varga weights, D = 5/4 diag(M), rho = 4/5).
// scale_mode 0: X scaled by 1; 1: block-preconditioner scaling of the
// (1,1)/(2,2) blocks (1/(sc_t H^gamma) for the first slabs*P columns, 1/(sc_t beta) after);
// 2: X scaled by `scale`.
template <typename T>
struct ChebArgs {
  const T* B; T* X; T* tmpA; T* tmpB;
  int64_t ncols; int n1; int64_t n; int steps; T mass;
  int scale_mode; int P; int slabs; int nt; T tau; T beta; T gamma;
  T scale;
};
template <typename T>
cudaError_t launch_cheb(const ChebArgs<T>& a, cudaStream_t st);

// Exact mass solve (the direct alternative to the Chebyshev semi-iteration): X = M^{-1} B on
// a.ncols columns with M = M1 (x) M1 on the uniform grid, M1 = (h/6) tridiag(1, 4, 1), by
// the square-root-free Cholesky factors of M1 (subdiagonal l, reciprocal pivots id; n1
// entries) along y and then along x; the scaling of a.scale_mode as for launch_cheb.
template <typename T>
cudaError_t launch_mass_exact(const ChebArgs<T>& a, const T* l, const T* id, cudaStream_t st);

// Multigrid level kernels on batches of columns stored contiguously [b][node].
struct Stencil { double diag, edge, corner; };
template <typename T>
cudaError_t launch_smooth(const T* b, const T* xin, T* xout, int64_t B, int n1, Stencil s, T omega,
                          T* acc, int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st);
template <typename T>
cudaError_t launch_residual(const T* b, const T* x, T* r, int64_t B, int n1, Stencil s, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict(const T* r, T* bc, int64_t B, int n1f, cudaStream_t st);
template <typename T>
cudaError_t launch_prolong_add(const T* xc, T* xf, int64_t B, int n1f, cudaStream_t st);
template <typename T>
cudaError_t launch_scale(const T* b, T* x, int64_t cnt, T a, cudaStream_t st);

// Levels handled by the one-CTA-per-column V-cycle: L.n1[0] (finest handled)
// down to a single node, with their 9-point stencils.
struct FusedLevels { int nlev; int n1[13]; double diag[13], edge[13], corner[13]; };
// Cluster V-cycle: one thread-block cluster of C CTAs per column; the first nd
// levels are split into C horizontal bands (halo rows through distributed shared
// memory), the remaining small levels are solved redundantly in every CTA.
struct ClusterLevels { int nlev; int nd; int n1[13]; double diag[13], edge[13], corner[13]; };
size_t vcycle_cluster_smem(const ClusterLevels& L, int C, int esize);
template <typename T>
cudaError_t launch_vcycle_cluster(const T* b, T* x, int64_t B, const ClusterLevels& L, int C, T omega, int nu,
                                  T* acc, int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st);

// Full-hierarchy V-cycle (top level read from global memory, register-blocked
// sweeps, 1024 threads): usable when vcycle_full_fits(L, sizeof(T)).
// Column layouts beyond the compact [column][node] one: with b_L > 0 right-hand-side
// column c is read at b + (c / b_L) b_ss + (c % b_L) n; with acc the result of column c
// goes to acc + (c / acc_L) acc_ss + (acc_col0 + c % acc_L) n, added (acc_add) or stored.
struct VColumns { int64_t b_ss = 0; int b_L = 0; int acc_add = 1; };
bool vcycle_full_fits(const FusedLevels& L, int esize);
// Merged launches of the fused V-cycle over members with the same grid: member g's
// right-hand sides, outputs and level stencils in the CTAs of columns [g*per, (g+1)*per).
struct VtMulti {
  int ng = 1;
  int64_t per = 0;
  const void* b[kMaxGroup]; void* x[kMaxGroup]; void* acc[kMaxGroup];
  double diag[kMaxGroup][13], edge[kMaxGroup][13], corner[kMaxGroup][13];
};
template <typename T>
cudaError_t launch_vcycle_full_group(const T* const* b, T* const* x, T* const* acc, const FusedLevels* L, int ng,
                                     int64_t B, T omega, int nu, int64_t acc_ss, int acc_L, int acc_col0,
                                     cudaStream_t st, VColumns cols = VColumns());
template <typename T>
cudaError_t launch_vcycle_full(const T* b, T* x, int64_t B, const FusedLevels& L, T omega, int nu,
                               T* acc, int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st,
                               VColumns cols = VColumns());

// Exact mean solves by fast diagonalisation on the tensor cores (spectral.cu), float32,
// for grids of n1 = 63 and 127 interior nodes per side: the V-cycle's column conventions,
// the stencil (d, e, c) of the mean operator, and the constant image spectral_image(n1)
// (16-byte aligned device copy).  spectral_take_error reports (and clears) a bounded wait
// that ran out in one of its launches.
bool spectral_mean_supported(int n1);
size_t spectral_image_bytes(int n1);
std::vector<uint8_t> spectral_image(int n1);
// prec: 0, the exact form (both factors of every product split into two bfloat16 terms), is
// the only one launched; other values return cudaErrorInvalidValue.
cudaError_t launch_spectral_mean(const float* b, float* x, int64_t B, int n1, const void* img, double d, double e,
                                 double c, float* acc, int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st,
                                 VColumns cols = VColumns(), int prec = 0);
// Merged launches over members with the same grid: member g's right-hand sides b[g], outputs
// (x[g], or acc[g] with the shared strides) and mean-operator stencil (d, e, c) = stencil[g].
struct SpecMulti {
  int ng = 1;
  const float* b[kMaxGroup]; float* x[kMaxGroup]; float* acc[kMaxGroup];
  float l0[kMaxGroup], l1[kMaxGroup], l2[kMaxGroup];
};
// Column scaling of the solution (the mass blocks of the preconditioner), as launch_cheb's
// scale_mode: 1 scales column col by 1 / s with the block, time-weight and H^gamma factors of
// the mass blocks, 2 by the uniform factor `scale`, 0 not at all.
struct SpecScale {
  int mode = 0;                  // 0 none, 1 the mass blocks' factors, 2 the uniform factor `scale`
  int P = 1, slabs = 1, nt = 0;
  float tau = 1.0f, beta = 1.0f, gamma = 0.0f, scale = 1.0f;
};
// X = s M^{-1} B for ncols contiguous columns: the exact mass solve by the same fast
// diagonalisation (M = M1 (x) M1, stencil (16, 4, 1) h^2 / 36).
cudaError_t launch_spectral_mass(const float* B, float* X, int64_t ncols, int n1, const void* img, double h2_36,
                                 const SpecScale& sc, cudaStream_t st);
cudaError_t launch_spectral_mean_group(const float* const* b, float* const* x, float* const* acc,
                                       const double (*stencil)[3], int ng, int64_t B, int n1, const void* img,
                                       int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st,
                                       VColumns cols = VColumns());
cudaError_t spectral_take_error(bool* failed, cudaStream_t st);

// Krylov kernels.  Reductions are deterministic: fixed grid, fixed order.
constexpr int kDotBlocks = 608;
template <typename T>
cudaError_t launch_dot_partial(const T* a, const T* b, int64_t n, double* partial, cudaStream_t st);
cudaError_t launch_sum_partials(const double* partial, double* out, cudaStream_t st);

// MINRES scalar state (float64, device resident)
struct MinresState {
  double beta, beta_prev, beta1, eta;
  double c_m1, s_m1, c_m2, s_m2;
  double alpha, eps, delta, rho, c, s;
  double est, target;
  double coef_v, coef_vp, coef_q;      // coefficients of the v-recurrence
  double w_q, w_m1, w_m2, x_w;         // coefficients of the w/x updates
  double dot;                          // last reduced dot
  int flag;                            // 0 running, 1 est<=target, 2 breakdown(beta=0), 3 not SPD, 4 NaN
  int iter;
  int wx_pending;                      // 1: the w/x update of the last rotation is still to be applied
};
cudaError_t launch_minres_init(MinresState* s, const double* partial, double target, cudaStream_t st);
cudaError_t launch_minres_alpha(MinresState* s, const double* partial, cudaStream_t st);
cudaError_t launch_minres_rotate(MinresState* s, const double* partial, cudaStream_t st);
// v_new (in place over v_prev) = Kz*coef_q - v*coef_v - v_prev*coef_vp
template <typename T>
cudaError_t launch_minres_v(const T* Kz, const T* v, T* vprev, int64_t n, const MinresState* s, cudaStream_t st);
// w_new (over w_m2) = z*w_q - w_m1*w_m1c - w_m2*w_m2c ; x += x_w * w_new
// (nothing when s->wx_pending is 0: no rotation since the start or since the last update)
template <typename T, typename TX>
cudaError_t launch_minres_wx(const T* z, const T* wm1, T* wm2, TX* x, int64_t n, const MinresState* s,
                             cudaStream_t st);

// FGMRES scalar state (float64, device resident): the cycle's Hessenberg matrix after
// its Givens rotations (column-major, leading dimension kFgmresMax + 1), the rotations,
// the rotated right-hand side g, the Gram-Schmidt coefficients of the current column
// and the least-squares solution y.
constexpr int kFgmresMax = 512;
struct FgmresState {
  double beta;                         // ||r|| at the start of the cycle
  double target, est;                  // stopping target and estimate |g_{j+1}| / ||b||
  double bnorm;                        // ||b|| of the solve (estimates are relative to it)
  double hnext;                        // ||w|| of the last column before its rotation
  int j;                               // columns of the cycle so far
  int flag;                            // 0 running, 1 est <= target, 2 breakdown, 4 NaN
  double h[kFgmresMax + 1], h2[kFgmresMax + 1];
  double cs[kFgmresMax], sn[kFgmresMax], g[kFgmresMax + 1], y[kFgmresMax];
  double H[(kFgmresMax + 1) * kFgmresMax];
};
// h[0..count) (or h2 with second = 1) = V_i . w for the count = s->j + 1 basis vectors
// V_i = V + i * ldv (n entries each); partial needs count * kDotBlocks doubles.
template <typename T>
cudaError_t launch_fgmres_multidot(const T* V, int64_t ldv, const T* w, int64_t n, FgmresState* s, int second,
                                   double* partial, cudaStream_t st);
// w -= sum_i c_i V_i over the s->j + 1 basis vectors, c = s->h (second = 0) or s->h2 (1);
// with add = 1 instead x += sum_i y_i V_i over the s->j columns (the solution update).
template <typename T, typename TX>
cudaError_t launch_fgmres_axpy(TX* w, const T* V, int64_t ldv, int64_t n, const FgmresState* s, int mode,
                               cudaStream_t st);
// start of a cycle from the reduced partials of r . r: beta, g = (beta, 0, ...), j = 0
cudaError_t launch_fgmres_start(FgmresState* s, const double* partial, double target, double bnorm,
                                cudaStream_t st);
// column j of H from h + h2 and the norm partials of w, rotations, estimate and flag; j += 1
cudaError_t launch_fgmres_rotate(FgmresState* s, const double* partial, cudaStream_t st);
// y from the triangular system of the cycle's s->j columns
cudaError_t launch_fgmres_solve_y(FgmresState* s, cudaStream_t st);
// out = in * (1 / s->beta) (which = 0) or in * (1 / s->hnext) (which = 1)
template <typename T>
cudaError_t launch_fgmres_scale(const T* in, T* out, int64_t n, const FgmresState* s, int which, cudaStream_t st);

// elementwise helpers
template <typename TA, typename TB>
cudaError_t launch_convert(const TA* a, TB* b, int64_t n, cudaStream_t st);
// y = a - b (float64); y may alias a
cudaError_t launch_sub(const double* a, const double* b, double* y, int64_t n, cudaStream_t st);
// x += (double) d
template <typename T>
cudaError_t launch_add_to(const T* d, double* x, int64_t n, cudaStream_t st);
// x += a * (double) d
cudaError_t launch_add_scaled(const float* d, double* x, int64_t n, double a, cudaStream_t st);
// y = a * x (scaling into float32 with a float64 scale)
cudaError_t launch_scale_to32(const double* x, float* y, int64_t n, double a, cudaStream_t st);
template <typename T>
cudaError_t launch_fill(T* x, int64_t n, T v, cudaStream_t st);

}  // namespace sgoc
