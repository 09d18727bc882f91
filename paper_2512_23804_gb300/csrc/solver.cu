// Solver orchestration: KKT products, block preconditioner (Chebyshev mass
// blocks, hierarchical Gauss-Seidel Schur block with batched V-cycles),
// preconditioned MINRES, float32/float64 iterative refinement and the ABI hooks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <functional>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "sgoc_internal.h"

namespace sgoc {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename T> static const T* kap_of(const sgoc_problem* pb);
template <> const double* kap_of<double>(const sgoc_problem* pb) { return pb->dev.kap64; }
template <> const float* kap_of<float>(const sgoc_problem* pb) { return pb->dev.kap32; }
template <typename T> static const T* nbrc_of(const sgoc_problem* pb);
template <> const double* nbrc_of<double>(const sgoc_problem* pb) { return pb->dev.nbr_c64; }
template <> const float* nbrc_of<float>(const sgoc_problem* pb) { return pb->dev.nbr_c32; }

static sgoc_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SGOC_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SGOC_ERR_CUDA;
}
#define SGOC_LAUNCH(...) SGOC_TRY(cuda_status((__VA_ARGS__), #__VA_ARGS__))

// Bump allocator over a caller-provided buffer (the library never allocates).
struct Carver {
  char* base; size_t cap; size_t off = 0; bool dry;
  Carver(void* b, size_t c, bool dry_run) : base(static_cast<char*>(b)), cap(c), dry(dry_run) {}
  template <typename T> T* take(size_t count) {
    char* p = dry ? nullptr : base + off;
    off = align256(off + count * sizeof(T));
    return reinterpret_cast<T*>(p);
  }
  bool ok() const { return dry || off <= cap; }
};

// Where the fused V-cycle starts and which kernel runs it.  Levels above lf use
// grid-wide level kernels.  float32: up to 127 x 127 interior nodes the whole
// hierarchy fits one CTA's shared memory (34 us per 127 x 127 cycle, faster than
// a 4-CTA cluster per column, 43 us); 255 x 255 takes an 8-CTA cluster (no single
// CTA holds it).  float64 runs at 1/64 of the float32 rate on this GPU: one CTA
// only up to 15 x 15, clusters of 2-8 CTAs for 31..127 so that each column's
// cycle is spread over several SMs.
struct VPlan { int lf = 0; bool cluster = false; int C = 1; int nd = 0; };

static VPlan plan_vcycle(const sgoc_problem* pb, int esize) {
  VPlan v;
  const int nl = int(pb->levels.size());
  for (int l = 0; l < nl; ++l) {
    const int n1 = pb->levels[l].n1;
    const int single_max = esize == 4 ? 127 : 15;
    const int cluster_max = esize == 4 ? 255 : 127;
    const int band0 = esize == 4 ? 32 : 16;
    const bool cluster_ok = n1 >= 31 && n1 <= cluster_max;
    const int C = (n1 + 1) / band0;
    const bool prefer_cluster = cluster_ok && (n1 > single_max || esize == 8);
    if (n1 <= single_max && !prefer_cluster) { v.lf = l; v.cluster = false; return v; }
    if (cluster_ok) {
      v.lf = l; v.cluster = true; v.C = C;
      v.nd = 0;
      for (int q = l; q < nl && (pb->levels[q].n1 + 1) / v.C >= 8; ++q) ++v.nd;
      return v;
    }
  }
  v.lf = nl - 1;
  return v;
}

int level_columns_max(const sgoc_problem* pb) {
  int m = 1;
  for (int d = 0; d <= pb->p; ++d) m = std::max(m, pb->off[d + 1] - pb->off[d]);
  return m;
}

// Preconditioner workspace of one precision.
template <typename T>
struct PrecWS {
  T* W1 = nullptr; T* W2 = nullptr;      // Schur-block intermediates (F each)
  T* chebA = nullptr; T* chebB = nullptr; // 2F each
  T* RH = nullptr;                       // hGS right-hand side of one level, all slabs
  std::vector<T*> lx, lt, lb;            // multigrid level arrays
};

template <typename T>
static void carve_prec(const sgoc_problem* pb, Carver& c, PrecWS<T>& w) {
  const size_t F = size_t(pb->F);
  w.W1 = c.template take<T>(F);
  w.W2 = c.template take<T>(F);
  w.chebA = c.template take<T>(2 * F);
  w.chebB = c.template take<T>(2 * F);
  const size_t B = size_t(pb->slabs) * level_columns_max(pb);
  w.RH = c.template take<T>(B * pb->n);
  const int nl = int(pb->levels.size());
  w.lx.assign(nl, nullptr); w.lt.assign(nl, nullptr); w.lb.assign(nl, nullptr);
  const int lf = plan_vcycle(pb, sizeof(T)).lf;
  for (int l = 0; l <= lf; ++l) {
    const size_t nlv = size_t(pb->levels[l].n);
    w.lx[l] = c.template take<T>(B * nlv);
    if (l < lf) w.lt[l] = c.template take<T>(B * nlv);
    if (l > 0) w.lb[l] = c.template take<T>(B * nlv);
  }
}

size_t precond_workspace_bytes(const sgoc_problem* pb, int esize) {
  Carver c(nullptr, 0, true);
  if (esize == 8) { PrecWS<double> w; carve_prec(pb, c, w); }
  else { PrecWS<float> w; carve_prec(pb, c, w); }
  return c.off;
}

// ---------------------------------------------------------------- V-cycle --
// One V(nu, nu) cycle for B columns of rhs `b` (compact [col][node] at level 0).
// With acc != nullptr the correction is added to the chaos columns of V
// (column col of the batch is slab col / acc_L, chaos column acc_col0 + col % acc_L).
// cols: strided right-hand side / stored strided output (VColumns), on the single-CTA path only
// With the exact mean solves (opt.mean_solve = 1) the same call is the exact solve by fast
// diagonalisation on the tensor cores (float32), with the same column conventions.
template <typename T>
static sgoc_status vcycle(const sgoc_problem* pb, PrecWS<T>& w, const T* b, T* xout, int64_t B, T* acc,
                          int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st, VColumns cols = VColumns()) {
  if (pb->opt.mean_solve != 0) {
    if constexpr (std::is_same<T, float>::value) {
      const Level& L0 = pb->levels[0];
      SGOC_LAUNCH(launch_spectral_mean(b, xout, B, pb->n1, pb->dev.spec_img, L0.diag, L0.edge, L0.corner, acc,
                                       acc_ss, acc_L, acc_col0, st, cols, pb->opt.mean_solve - 1));
      return SGOC_OK;
    } else {
      set_error("exact mean solves are float32 only");
      return SGOC_ERR_UNSUPPORTED;
    }
  }
  const int nl = int(pb->levels.size());
  const T om = T(pb->opt.omega);
  const int nu = pb->opt.nu_pre;
  const VPlan vp = plan_vcycle(pb, sizeof(T));
  const int lf = vp.lf;
  FusedLevels FL;
  ClusterLevels CL;
  FL.nlev = CL.nlev = nl - lf;
  CL.nd = vp.nd;
  for (int l = lf; l < nl; ++l) {
    FL.n1[l - lf] = CL.n1[l - lf] = pb->levels[l].n1;
    FL.diag[l - lf] = CL.diag[l - lf] = pb->levels[l].diag;
    FL.edge[l - lf] = CL.edge[l - lf] = pb->levels[l].edge;
    FL.corner[l - lf] = CL.corner[l - lf] = pb->levels[l].corner;
  }
  if (!vp.cluster && !vcycle_full_fits(FL, sizeof(T))) { set_error("internal: V-cycle level does not fit"); return SGOC_ERR_UNSUPPORTED; }
  if ((cols.b_L > 0 || !cols.acc_add) && (lf != 0 || vp.cluster)) {
    set_error("internal: strided V-cycle columns need the single-CTA cycle");
    return SGOC_ERR_UNSUPPORTED;
  }
  auto fused = [&](const T* bb, T* xx, T* ac, int64_t ss, int aL, int ac0) -> cudaError_t {
    if (vp.cluster) return launch_vcycle_cluster<T>(bb, xx, B, CL, vp.C, om, nu, ac, ss, aL, ac0, st);
    return launch_vcycle_full<T>(bb, xx, B, FL, om, nu, ac, ss, aL, ac0, st, cols);
  };
  if (lf == 0) {
    SGOC_LAUNCH(fused(b, xout, acc, acc_ss, acc_L, acc_col0));
    return SGOC_OK;
  }
  // level-wise descent down to lf
  std::vector<T*> xcur(nl, nullptr), spare(nl, nullptr);
  std::vector<const T*> bl(nl, nullptr);
  bl[0] = b;
  for (int l = 0; l < lf; ++l) {
    const Level& L = pb->levels[l];
    Stencil s{L.diag, L.edge, L.corner};
    T* xa = w.lx[l];
    T* xb = w.lt[l];
    T* cur = nullptr;
    for (int sw = 0; sw < nu; ++sw) {
      T* dst = (cur == xa) ? xb : xa;
      SGOC_LAUNCH(launch_smooth<T>(bl[l], cur, dst, B, L.n1, s, om, nullptr, 0, 1, 0, st));
      cur = dst;
    }
    if (!cur) { SGOC_LAUNCH(launch_fill<T>(xa, B * L.n, T(0), st)); cur = xa; }
    T* sp = (cur == xa) ? xb : xa;
    SGOC_LAUNCH(launch_residual<T>(bl[l], cur, sp, B, L.n1, s, st));
    SGOC_LAUNCH(launch_restrict<T>(sp, w.lb[l + 1], B, L.n1, st));
    bl[l + 1] = w.lb[l + 1];
    xcur[l] = cur; spare[l] = sp;
  }
  SGOC_LAUNCH(fused(bl[lf], w.lx[lf], (T*)nullptr, 0, 1, 0));
  T* xc = w.lx[lf];
  for (int l = lf - 1; l >= 0; --l) {
    const Level& L = pb->levels[l];
    Stencil s{L.diag, L.edge, L.corner};
    T* cur = xcur[l];
    T* sp = spare[l];
    SGOC_LAUNCH(launch_prolong_add<T>(xc, cur, B, L.n1, st));
    for (int sw = 0; sw < nu; ++sw) {
      const bool last = (sw == nu - 1);
      if (l == 0 && last) {
        SGOC_LAUNCH(launch_smooth<T>(bl[l], cur, acc ? nullptr : xout, B, L.n1, s, om, acc, acc_ss, acc_L,
                                     acc_col0, st));
        cur = nullptr;
      } else {
        SGOC_LAUNCH(launch_smooth<T>(bl[l], cur, sp, B, L.n1, s, om, nullptr, 0, 1, 0, st));
        std::swap(cur, sp);
      }
    }
    if (l == 0 && nu == 0) {
      // no smoothing: hand the corrected x over
      if (acc) return set_error("nu = 0 with accumulation is not supported"), SGOC_ERR_INVALID_ARG;
      SGOC_LAUNCH(launch_scale<T>(cur, xout, B * L.n, T(1), st));
    }
    xc = cur;
  }
  return SGOC_OK;
}

// number of (output column, neighbour) pairs with KL index < kmax
static double deg_sum(const sgoc_problem* pb, int out0, int out1, int kmax) {
  double s = 0;
  for (int b = out0; b < out1; ++b)
    for (int e = pb->nbr_ptr[b]; e < pb->nbr_ptr[b + 1]; ++e)
      if (pb->nbr_k[e] < kmax) s += 1;
  return s;
}

// -------------------------------------------------------------------- hGS --
// V = Z_hGS^{-1} R over `slabs` panels (Alg. 1, correction form, palindromic level order).
// The slot table of an SG launch shape (two-phase kernel).
template <typename T>
static void set_utab(SGArgs<T>& g, const UTab& u) {
  g.u_mb = u.d_mb; g.u_diag = u.d_diag; g.u_eptr = u.d_eptr; g.u_e32 = u.d_e32;
  g.u_nslots = u.nslots; g.u_nent = u.nent;
}

// the chaos degree and coupling values the register SG kernel takes (Legendre chaos only)
template <typename T>
static void set_legendre(SGArgs<T>& g, const sgoc_problem* pb) {
  g.legendre_p = pb->sgr_ok && pb->p <= 10 ? pb->p : -1;
  for (int j = 0; j < 11; ++j) g.cup[j] = T(j < pb->p ? legendre_coupling(j) : 0.0);
}

// SG launch of the hGS visit of level d: rhs of the level's columns (correction form)
template <typename T>
static SGArgs<T> hgs_args(const sgoc_problem* pb, PrecWS<T>& w, const T* R, T* V, int slabs, int d) {
  const int P = pb->P, p = pb->p;
  const int64_t n = pb->n, ps = int64_t(P) * n;
  const bool time = pb->nt > 0;
  const T cK = T(time ? pb->tau : 1.0);                 // multiplies K_0 .. K_M
  const T cM = T(time ? 1.0 + pb->tau * pb->s : pb->s); // multiplies M in the mean operator
  const int a0 = pb->off[d], a1 = pb->off[d + 1], L = a1 - a0;
  SGArgs<T> g{};
  g.X = V; g.xs = ps;
  g.Y = w.RH; g.ys = int64_t(L) * n; g.ycol0 = a0;
  g.R = R; g.rs = ps; g.rcol0 = 0;
  g.n1 = pb->n1; g.n = n; g.nx = pb->nx; g.M = pb->nterms - 1;
  g.out0 = a0; g.out1 = a1;
  // the levels coupled to level d by a kept term: within lev_dist of d (1 for Legendre)
  g.in0 = pb->off[std::max(0, d - pb->lev_dist)];
  g.in1 = pb->off[std::min(p + 1, d + pb->lev_dist + 1)];
  g.kmax = pb->r; g.nslabs = slabs;
  g.c0 = -cK; g.c1 = -cK; g.cm = -cM; g.cr = T(1); g.cy = T(0);
  g.mass = T(pb->mass_h2_36);
  g.kap = kap_of<T>(pb);
  g.nbr_ptr = pb->dev.nbr_ptr; g.nbr_alpha = pb->dev.nbr_alpha; g.nbr_k = pb->dev.nbr_k; g.nbr_c = nbrc_of<T>(pb);
  g.nbr_end = pb->r == pb->nterms ? pb->dev.nbr_end_all : pb->dev.nbr_end_r;
  g.deg_sum = deg_sum(pb, a0, a1, pb->r);
  g.nnz_out = pb->nbr_ptr[a1] - pb->nbr_ptr[a0];
  set_utab(g, pb->utabs[1 + d]);
  set_legendre(g, pb);
  return g;
}

// The first (ascending) visit of level d: levels d and above are still zero, so the right-hand
// side is R_(d) minus the couplings to level d - 1 only (downward neighbour table), without the
// level's own kappa_0 and mass terms.  The same values as hgs_args on the zero-padded levels.
template <typename T>
static SGArgs<T> hgs_args_first(const sgoc_problem* pb, PrecWS<T>& w, const T* R, T* V, int slabs, int d) {
  SGArgs<T> g = hgs_args<T>(pb, w, R, V, slabs, d);
  const int a0 = pb->off[d], a1 = pb->off[d + 1];
  g.in0 = pb->off[std::max(0, d - pb->lev_dist)];
  g.in1 = a0;
  g.no_own = 1;
  g.c0 = T(0); g.cm = T(0);
  g.nbr_ptr = pb->dev.dn_ptr; g.nbr_alpha = pb->dev.dn_alpha; g.nbr_k = pb->dev.dn_k;
  g.nbr_c = std::is_same<T, double>::value ? reinterpret_cast<const T*>(pb->dev.dn_c64)
                                           : reinterpret_cast<const T*>(pb->dev.dn_c32);
  g.nbr_end = pb->r == pb->nterms ? pb->dev.dn_ptr + 1 : pb->dev.dn_end_r;
  g.nnz_out = pb->dn_ptr[a1] - pb->dn_ptr[a0];
  double deg = 0;
  for (int b = a0; b < a1; ++b)
    for (int e = pb->dn_ptr[b]; e < pb->dn_ptr[b + 1]; ++e) deg += pb->dn_k[e] < pb->r ? 1 : 0;
  g.deg_sum = deg;
  set_utab(g, pb->utabs[2 + pb->p + d]);
  return g;
}

template <typename T>
static sgoc_status hgs(const sgoc_problem* pb, PrecWS<T>& w, const T* R, T* V, int slabs, cudaStream_t st) {
  const int P = pb->P, p = pb->p;
  const int64_t n = pb->n, ps = int64_t(P) * n;
  // The first visit of each level stores its correction (levels are never read before their
  // first visit), so V needs no zero fill: with one slab a level's columns are contiguous;
  // with several, the single-CTA V-cycle stores into the strided layout.  Otherwise (several
  // slabs on the cluster or level-wise cycle) the corrections are added into a zeroed V.
  const bool one = slabs == 1;
  const VPlan vp = plan_vcycle(pb, sizeof(T));
  const bool strided = vp.lf == 0 && !vp.cluster;
  if (!one && !strided) SGOC_LAUNCH(launch_fill<T>(V, slabs * ps, T(0), st));
  // palindromic sweep 0, 1, ..., p, ..., 1, 0: the first visit of each level, then the returns
  for (int step = 0; step < 2 * p + 1; ++step) {
    const bool first = step <= p;
    const int d = first ? step : 2 * p - step;
    const int a0 = pb->off[d], L = pb->off[d + 1] - a0;
    // the first visit of level 0 has no couplings: its right-hand side is R_0 itself, read in
    // place by the V-cycle (a contiguous column with one slab, slab-strided columns otherwise)
    const T* rhs = w.RH;
    VColumns cols;
    if (first && d == 0 && (one || strided)) {
      rhs = R;
      if (!one) { cols.b_L = 1; cols.b_ss = ps; }
    } else {
      SGOC_LAUNCH(launch_sg<T>(first ? hgs_args_first<T>(pb, w, R, V, slabs, d) : hgs_args<T>(pb, w, R, V, slabs, d),
                               st));
    }
    if (first && one) {
      SGOC_TRY(vcycle<T>(pb, w, rhs, V + int64_t(a0) * n, L, nullptr, 0, 1, 0, st, cols));
    } else {
      if (first && strided) cols.acc_add = 0;       // store (V was not zero-filled)
      SGOC_TRY(vcycle<T>(pb, w, rhs, nullptr, int64_t(slabs) * L, V, ps, L, a0, st, cols));
    }
  }
  return SGOC_OK;
}

// ------------------------------------------------------------- merged hGS --
// One hGS sweep (as hgs above) for several problems of one shape at once: each level
// visit is one SG launch and one V-cycle launch over all members' columns (merged
// launches: member g's operands, coefficient data and mean-operator stencils in its
// own CTAs), so a visit of a level with L columns fills g * L * slabs CTAs.  Every
// member's arithmetic is that of hgs() on its own, so the results are bitwise equal.
// Mergeable: same grid, chaos levels, truncation, slabs, sweep counts, damping and a
// single-CTA fused V-cycle from the finest level (otherwise the members' sweeps run
// one after the other).
template <typename T>
struct HgsMember { const sgoc_problem* pb; PrecWS<T>* w; const T* R; T* V; };

static FusedLevels fused_levels_of(const sgoc_problem* pb, int lf) {
  FusedLevels FL{};
  const int nl = int(pb->levels.size());
  FL.nlev = nl - lf;
  for (int l = lf; l < nl; ++l) {
    FL.n1[l - lf] = pb->levels[l].n1;
    FL.diag[l - lf] = pb->levels[l].diag;
    FL.edge[l - lf] = pb->levels[l].edge;
    FL.corner[l - lf] = pb->levels[l].corner;
  }
  return FL;
}

static bool same_shape(const sgoc_problem* a, const sgoc_problem* b) {
  return a->nx == b->nx && a->M == b->M && a->p == b->p && a->slabs == b->slabs && a->r == b->r &&
         a->chaos == b->chaos && a->nterms == b->nterms &&
         a->opt.precision == b->opt.precision && a->opt.nu_pre == b->opt.nu_pre &&
         a->opt.nu_post == b->opt.nu_post && a->opt.omega == b->opt.omega &&
         a->opt.cheb_steps == b->opt.cheb_steps && a->opt.mean_solve == b->opt.mean_solve &&
         (a->nt > 0) == (b->nt > 0);
}

template <typename T>
static bool hgs_mergeable(const std::vector<HgsMember<T>>& ms) {
  if (ms.size() < 2 || ms.size() > size_t(kMaxGroup)) return false;
  const int mean = ms[0].pb->opt.mean_solve;
  for (const auto& m : ms)
    if (!same_shape(m.pb, ms[0].pb) || m.pb->opt.mean_solve != mean) return false;
  if (mean != 0) return std::is_same<T, float>::value;   // exact mean solves: one merged launch per visit
  const VPlan vp = plan_vcycle(ms[0].pb, sizeof(T));
  return vp.lf == 0 && !vp.cluster;
}

// the mean solves of one hGS level visit for every member (merged launches): the V-cycle, or
// the exact solve by fast diagonalisation
template <typename T>
static sgoc_status mean_group(const std::vector<HgsMember<T>>& ms, const T* const* rhs, T* const* xo, T* const* acc,
                              const FusedLevels* FL, int64_t B, int64_t acc_ss, int acc_L, int acc_col0,
                              cudaStream_t st, VColumns cols) {
  const sgoc_problem* pb = ms[0].pb;
  const int ng = int(ms.size());
  if (pb->opt.mean_solve != 0) {
    if constexpr (std::is_same<T, float>::value) {
      double sten[kMaxGroup][3];
      for (int g = 0; g < ng; ++g) {
        const Level& L0 = ms[g].pb->levels[0];
        sten[g][0] = L0.diag; sten[g][1] = L0.edge; sten[g][2] = L0.corner;
      }
      SGOC_LAUNCH(launch_spectral_mean_group(rhs, xo, acc, sten, ng, B, pb->n1, pb->dev.spec_img, acc_ss, acc_L,
                                             acc_col0, st, cols));
      return SGOC_OK;
    }
    set_error("exact mean solves are float32 only");
    return SGOC_ERR_UNSUPPORTED;
  }
  SGOC_LAUNCH(launch_vcycle_full_group<T>(rhs, xo, acc, FL, ng, B, T(pb->opt.omega), pb->opt.nu_pre, acc_ss, acc_L,
                                          acc_col0, st, cols));
  return SGOC_OK;
}

template <typename T>
static sgoc_status hgs_multi(const std::vector<HgsMember<T>>& ms, int slabs, cudaStream_t st) {
  if (!hgs_mergeable(ms)) {
    for (const auto& m : ms) SGOC_TRY(hgs<T>(m.pb, *m.w, m.R, m.V, slabs, st));
    return SGOC_OK;
  }
  const int ng = int(ms.size());
  const sgoc_problem* pb = ms[0].pb;
  const int P = pb->P, p = pb->p;
  const int64_t n = pb->n, ps = int64_t(P) * n;
  const bool one = slabs == 1;            // the single-CTA cycle stores strided columns otherwise
  FusedLevels FL[kMaxGroup];
  if (pb->opt.mean_solve == 0)
    for (int g = 0; g < ng; ++g) FL[g] = fused_levels_of(ms[g].pb, 0);
  for (int step = 0; step < 2 * p + 1; ++step) {
    const bool first = step <= p;
    const int d = first ? step : 2 * p - step;
    const int a0 = pb->off[d], L = pb->off[d + 1] - a0;
    const T* rhs[kMaxGroup];
    T* xo[kMaxGroup];
    T* acc[kMaxGroup];
    VColumns cols;
    if (first && d == 0) {
      for (int g = 0; g < ng; ++g) rhs[g] = ms[g].R;
      if (!one) { cols.b_L = 1; cols.b_ss = ps; }
    } else {
      SGArgs<T> a[kMaxGroup];
      for (int g = 0; g < ng; ++g) {
        a[g] = first ? hgs_args_first<T>(ms[g].pb, *ms[g].w, ms[g].R, ms[g].V, slabs, d)
                     : hgs_args<T>(ms[g].pb, *ms[g].w, ms[g].R, ms[g].V, slabs, d);
        rhs[g] = ms[g].w->RH;
      }
      SGOC_LAUNCH(launch_sg_group<T>(a, ng, st));
    }
    if (first && one) {
      for (int g = 0; g < ng; ++g) { xo[g] = ms[g].V + int64_t(a0) * n; acc[g] = nullptr; }
      SGOC_TRY(mean_group<T>(ms, rhs, xo, acc, FL, L, 0, 1, 0, st, cols));
    } else {
      if (first) cols.acc_add = 0;                  // store (V was not zero-filled)
      for (int g = 0; g < ng; ++g) { xo[g] = nullptr; acc[g] = ms[g].V; }
      SGOC_TRY(mean_group<T>(ms, rhs, xo, acc, FL, int64_t(slabs) * L, ps, L, a0, st, cols));
    }
  }
  return SGOC_OK;
}

// Independent pieces of one KKT product or preconditioner application run on two
// auxiliary streams (parallel branches when captured into a graph).
struct Fork {
  cudaStream_t s1 = nullptr, s2 = nullptr;
  cudaStream_t s3 = nullptr;            // the deferred MINRES w/x update beside the KKT product
  cudaEvent_t e[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

static sgoc_status fork_to(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  SGOC_CUDA_TRY(cudaEventRecord(ev, from));
  SGOC_CUDA_TRY(cudaStreamWaitEvent(to, ev, 0));
  pdl_fence(to);
  return SGOC_OK;
}

// -------------------------------------------------------------- KKT apply --
template <typename T>
static SGArgs<T> sg_full(const sgoc_problem* pb, const T* X, T* Y, T coef) {
  SGArgs<T> g{};
  const int64_t ps = int64_t(pb->P) * pb->n;
  g.X = X; g.xs = ps; g.Y = Y; g.ys = ps; g.ycol0 = 0;
  g.R = nullptr; g.rs = 0; g.rcol0 = 0;
  g.n1 = pb->n1; g.n = pb->n; g.nx = pb->nx; g.M = pb->nterms - 1;
  g.out0 = 0; g.out1 = pb->P; g.in0 = 0; g.in1 = pb->P;
  g.kmax = pb->nterms; g.nslabs = pb->slabs;
  g.c0 = coef; g.c1 = coef; g.cm = T(0); g.cr = T(0); g.cy = T(1);
  g.mass = T(pb->mass_h2_36);
  g.kap = kap_of<T>(pb);
  g.nbr_ptr = pb->dev.nbr_ptr; g.nbr_alpha = pb->dev.nbr_alpha; g.nbr_k = pb->dev.nbr_k; g.nbr_c = nbrc_of<T>(pb);
  g.nbr_end = pb->dev.nbr_end_all;
  g.deg_sum = double(pb->nbr_alpha.size());
  g.nnz_out = int(pb->nbr_alpha.size());
  set_utab(g, pb->utabs[0]);
  set_legendre(g, pb);
  return g;
}

template <typename T>
static MassArgs<T> mass_base(const sgoc_problem* pb, T* out) {
  MassArgs<T> m{};
  m.out = out; m.os = int64_t(pb->P) * pb->n;
  m.ncols = pb->P; m.col0 = 0; m.nslabs = pb->slabs; m.n1 = pb->n1; m.n = pb->n;
  m.mass = T(pb->mass_h2_36); m.cy = T(0); m.ar = T(0); m.gamma = T(pb->gamma); m.nt = pb->nt;
  m.nv = 0; m.R = nullptr; m.rs = 0;
  return m;
}

template <typename T>
static void mass_add(MassArgs<T>& m, const T* V, int shift, double a, int wflags, int64_t vs) {
  m.V[m.nv] = V; m.vs[m.nv] = vs; m.shift[m.nv] = shift; m.a[m.nv] = T(a); m.wflags[m.nv] = wflags;
  ++m.nv;
}

template <typename T>
static sgoc_status kkt_apply(const sgoc_problem* pb, const T* v, T* w, cudaStream_t st,
                             const Fork* f = nullptr) {
  const int64_t F = pb->F, ps = int64_t(pb->P) * pb->n;
  const T* y = v; const T* u = v + F; const T* lam = v + 2 * F;
  T* w1 = w; T* w2 = w + F; T* w3 = w + 2 * F;
  if (pb->nt == 0) {
    // w1 = M Y H^gamma - A Lambda ; w2 = beta M U + M Lambda ; w3 = -A Y + M U   (Eq. (stoch-system))
    // the three block rows are independent: rows 2 and 3 on the auxiliary streams
    cudaStream_t s2 = st, s3 = st;
    if (f) {
      SGOC_TRY(fork_to(st, f->s1, f->e[0]));
      SGOC_TRY(fork_to(st, f->s2, f->e[0]));
      s2 = f->s1; s3 = f->s2;
    }
    MassArgs<T> m1 = mass_base<T>(pb, w1); mass_add(m1, y, 0, 1.0, 1, ps);
    SGOC_LAUNCH(launch_mass<T>(m1, st));
    SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, lam, w1, T(-1)), st));
    MassArgs<T> m2 = mass_base<T>(pb, w2); mass_add(m2, u, 0, pb->beta, 0, ps); mass_add(m2, lam, 0, 1.0, 0, ps);
    SGOC_LAUNCH(launch_mass<T>(m2, s2));
    MassArgs<T> m3 = mass_base<T>(pb, w3); mass_add(m3, u, 0, 1.0, 0, ps);
    SGOC_LAUNCH(launch_mass<T>(m3, s3));
    SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, y, w3, T(-1)), s3));
    if (f) {
      SGOC_TRY(fork_to(f->s1, st, f->e[1]));
      SGOC_TRY(fork_to(f->s2, st, f->e[2]));
    }
    return SGOC_OK;
  }
  // time (Eq. (KKT:stoch-time-dependent)), A_t = I (x) (M_cal + tau A) - C (x) M_cal:
  // w1_t = tau D_t M Y_t H^g - (M L_t + tau A L_t - M L_{t+1})
  // w2_t = beta tau D_t M U_t + tau M L_t
  // w3_t = -(M Y_t + tau A Y_t - M Y_{t-1}) + tau M U_t
  const double tau = pb->tau;
  cudaStream_t s2 = st, s3 = st;
  if (f) {
    SGOC_TRY(fork_to(st, f->s1, f->e[0]));
    SGOC_TRY(fork_to(st, f->s2, f->e[0]));
    s2 = f->s1; s3 = f->s2;
  }
  MassArgs<T> m1 = mass_base<T>(pb, w1);
  mass_add(m1, y, 0, tau, 3, ps); mass_add(m1, lam, 0, -1.0, 0, ps); mass_add(m1, lam, 1, 1.0, 0, ps);
  SGOC_LAUNCH(launch_mass<T>(m1, st));
  SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, lam, w1, T(-tau)), st));
  MassArgs<T> m2 = mass_base<T>(pb, w2);
  mass_add(m2, u, 0, pb->beta * tau, 2, ps); mass_add(m2, lam, 0, tau, 0, ps);
  SGOC_LAUNCH(launch_mass<T>(m2, s2));
  MassArgs<T> m3 = mass_base<T>(pb, w3);
  mass_add(m3, y, 0, -1.0, 0, ps); mass_add(m3, y, -1, 1.0, 0, ps); mass_add(m3, u, 0, tau, 0, ps);
  SGOC_LAUNCH(launch_mass<T>(m3, s3));
  SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, y, w3, T(-tau)), s3));
  if (f) {
    SGOC_TRY(fork_to(f->s1, st, f->e[1]));
    SGOC_TRY(fork_to(f->s2, st, f->e[2]));
  }
  return SGOC_OK;
}

// The mass blocks 1 and 2: Chebyshev semi-iteration, or the exact solve (sgoc_options.mass_solve)
template <typename T> static const T* mass_l_of(const sgoc_problem* pb);
template <> const double* mass_l_of<double>(const sgoc_problem* pb) { return pb->dev.mass_l64; }
template <> const float* mass_l_of<float>(const sgoc_problem* pb) { return pb->dev.mass_l32; }
template <typename T> static const T* mass_id_of(const sgoc_problem* pb);
template <> const double* mass_id_of<double>(const sgoc_problem* pb) { return pb->dev.mass_id64; }
template <> const float* mass_id_of<float>(const sgoc_problem* pb) { return pb->dev.mass_id32; }

template <typename T>
static cudaError_t launch_mass_blocks(const sgoc_problem* pb, const ChebArgs<T>& c, cudaStream_t st) {
  if (pb->opt.mass_solve == 1) {
    // float32 on the grids of the tensor-core transform: the exact solve by fast diagonalisation
    if constexpr (std::is_same<T, float>::value) {
      if (pb->dev.spec_img != nullptr && c.scale_mode >= 0 && c.scale_mode <= 2) {
        SpecScale sc;
        sc.mode = c.scale_mode; sc.P = c.P; sc.slabs = c.slabs; sc.nt = c.nt;
        sc.tau = c.tau; sc.beta = c.beta; sc.gamma = c.gamma; sc.scale = c.scale;
        return launch_spectral_mass(c.B, c.X, c.ncols, pb->n1, pb->dev.spec_img, pb->mass_h2_36, sc, st);
      }
    }
    return launch_mass_exact<T>(c, mass_l_of<T>(pb), mass_id_of<T>(pb), st);
  }
  return launch_cheb<T>(c, st);
}

// ------------------------------------------------ coupled time Schur block --
// z = tau Z_bar^{-T} (D (x) M_gamma) Z_bar^{-1} r with Z_bar = I (x) Z~_t - C (x) M_cal (Eq. (S hat),
// Eq. (Z hat)): Z_bar x = r by forward substitution, Z~ x_t = r_t + M_cal x_{t-1}, and
// Z_bar^T z = w by backward substitution, Z~ z_t = w_t + M_cal z_{t+1}; each solve with the slab
// operator Z~ is one hGS sweep of one slab (Alg. 1), so the slabs run one after the other.
template <typename T>
static sgoc_status coupled_schur(const sgoc_problem* pb, PrecWS<T>& w, const T* r, T* z, cudaStream_t st) {
  const int nt = pb->nt;
  const int64_t ps = int64_t(pb->P) * pb->n;
  // one slab: out = R + M V  (every chaos column, no weights)
  auto coupled_rhs = [&](T* out, const T* R, const T* V) -> sgoc_status {
    MassArgs<T> m = mass_base<T>(pb, out);
    m.nslabs = 1;
    m.R = R; m.rs = ps; m.ar = T(1);
    mass_add(m, V, 0, 1.0, 0, ps);
    SGOC_LAUNCH(launch_mass<T>(m, st));
    return SGOC_OK;
  };
  for (int t = 0; t < nt; ++t) {                       // W1 = Z_bar^{-1} r
    const T* rhs = r;
    if (t > 0) {
      SGOC_TRY(coupled_rhs(w.W2 + t * ps, r + t * ps, w.W1 + (t - 1) * ps));
      rhs = w.W2 + t * ps;
    }
    SGOC_TRY(hgs<T>(pb, w, rhs, w.W1 + t * ps, 1, st));
  }
  MassArgs<T> m = mass_base<T>(pb, w.W2);               // W2 = tau (D (x) M_gamma) W1
  mass_add(m, w.W1, 0, pb->tau, 3, ps);
  SGOC_LAUNCH(launch_mass<T>(m, st));
  for (int t = nt - 1; t >= 0; --t) {                  // z = Z_bar^{-T} W2
    const T* rhs = w.W2 + t * ps;
    if (t + 1 < nt) {
      SGOC_TRY(coupled_rhs(w.W1 + t * ps, w.W2 + t * ps, z + (t + 1) * ps));
      rhs = w.W1 + t * ps;
    }
    SGOC_TRY(hgs<T>(pb, w, rhs, z + t * ps, 1, st));
  }
  return SGOC_OK;
}

// -------------------------------------------------------------------- hGSoc --
// The hGS preconditioner for the optimal control problem (Alg. 2-3) on slab t of r (every slab
// independently: Alg. 4), into z.  Levels 0, 1, ..., p, ..., 1, 0; at a visit of level d the
// level's three fields are overwritten by one solve with
//   P~ = blkdiag(sc M, beta sc M, (1/sc) A~ M^{-1} A~)     (sc = 1 steady, tau D_t in time mode)
// of R_(d) plus the truncated couplings to the other levels: Y from c K_k Lambda G_k, Lambda from
// c K_k Y G_k (c = 1, or tau); the U block has no coupling and is solved once.  First visits need
// the couplings to the level below only (the levels above are still zero): the downward table.
template <typename T>
static sgoc_status hgsoc_slab(const sgoc_problem* pb, PrecWS<T>& w, const T* r, T* z, int t, cudaStream_t st) {
  const int64_t F = pb->F, n = pb->n, ps = int64_t(pb->P) * n;
  const bool time = pb->nt > 0;
  const double sc = time ? pb->tau * pb->dweights[t] : 1.0;
  const T cK = T(time ? pb->tau : 1.0);
  const T* rY = r + t * ps; const T* rU = r + F + t * ps; const T* rL = r + 2 * F + t * ps;
  T* zY = z + t * ps; T* zU = z + F + t * ps; T* zL = z + 2 * F + t * ps;
  T* T1 = w.chebA;                       // Lambda solve intermediates (compact level columns)
  T* T2 = w.chebA + F;
  auto mass_solve = [&](const T* b, T* x, int ncols, double scale) -> sgoc_status {
    ChebArgs<T> c{};
    c.B = b; c.X = x; c.tmpA = w.chebB; c.tmpB = w.chebB + F;
    c.ncols = ncols; c.n1 = pb->n1; c.n = n; c.steps = pb->opt.cheb_steps;
    c.mass = T(pb->mass_h2_36); c.scale_mode = 2; c.scale = T(scale);
    c.P = ncols; c.slabs = 1; c.nt = 0;
    SGOC_LAUNCH(launch_mass_blocks<T>(pb, c, st));
    return SGOC_OK;
  };
  SGOC_TRY(mass_solve(rU, zU, pb->P, 1.0 / (pb->beta * sc)));
  const int p = pb->p;
  for (int step = 0; step < 2 * p + 1; ++step) {
    const bool first = step <= p;
    const int d = first ? step : 2 * p - step;
    const int a0 = pb->off[d], L = pb->off[d + 1] - a0;
    const T* bY = rY + int64_t(a0) * n;
    const T* bL = rL + int64_t(a0) * n;
    if (!(first && d == 0)) {
      for (int fld = 0; fld < 2; ++fld) {
        // fld 0: the Y right-hand side from Lambda; fld 1: the Lambda right-hand side from Y
        SGArgs<T> g = first ? hgs_args_first<T>(pb, w, fld == 0 ? rY : rL, fld == 0 ? zL : zY, 1, d)
                            : hgs_args<T>(pb, w, fld == 0 ? rY : rL, fld == 0 ? zL : zY, 1, d);
        g.no_own = 1; g.c0 = T(0); g.cm = T(0); g.c1 = cK; g.cr = T(1); g.cy = T(0);
        g.Y = fld == 0 ? w.W1 : w.W2; g.ycol0 = a0; g.ys = int64_t(L) * n;
        SGOC_LAUNCH(launch_sg<T>(g, st));
      }
      bY = w.W1; bL = w.W2;
    }
    SGOC_TRY(mass_solve(bY, zY + int64_t(a0) * n, L, 1.0 / sc));
    SGOC_TRY(vcycle<T>(pb, w, bL, T1, L, nullptr, 0, 1, 0, st));
    MassArgs<T> m = mass_base<T>(pb, T2);
    m.ncols = L; m.nslabs = 1; m.os = int64_t(L) * n;
    mass_add(m, T1, 0, sc, 0, int64_t(L) * n);
    SGOC_LAUNCH(launch_mass<T>(m, st));
    SGOC_TRY(vcycle<T>(pb, w, T2, zL + int64_t(a0) * n, L, nullptr, 0, 1, 0, st));
  }
  return SGOC_OK;
}

// ------------------------------------------------------ block preconditioner --
template <typename T>
static sgoc_status precond_apply(const sgoc_problem* pb, PrecWS<T>& w, const T* r, T* z, cudaStream_t st,
                                 const Fork* f = nullptr,
                                 const std::function<sgoc_status(cudaStream_t)>& before_cheb = nullptr) {
  const int64_t F = pb->F, ps = int64_t(pb->P) * pb->n;
  if (pb->opt.precond == 1) {                           // hGSoc (Alg. 2-3), slab by slab (Alg. 4)
    for (int t = 0; t < pb->slabs; ++t) SGOC_TRY(hgsoc_slab<T>(pb, w, r, z, t, st));
    return SGOC_OK;
  }
  // blocks 1, 2: Chebyshev on M, scaled by 1/(sc_t H^gamma) and 1/(sc_t beta)
  ChebArgs<T> c{};
  c.B = r; c.X = z; c.tmpA = w.chebA; c.tmpB = w.chebB;
  c.ncols = 2 * int64_t(pb->slabs) * pb->P; c.n1 = pb->n1; c.n = pb->n; c.steps = pb->opt.cheb_steps;
  c.mass = T(pb->mass_h2_36); c.scale_mode = 1; c.P = pb->P; c.slabs = pb->slabs; c.nt = pb->nt;
  c.tau = T(pb->tau); c.beta = T(pb->beta); c.gamma = T(pb->gamma);
  // blocks 1, 2 (Chebyshev) are independent of block 3: run them on an auxiliary stream
  cudaStream_t sc = st;
  if (f) { SGOC_TRY(fork_to(st, f->s1, f->e[3])); sc = f->s1; }
  if (before_cheb) SGOC_TRY(before_cheb(sc));       // work only the Chebyshev blocks wait for
  SGOC_LAUNCH(launch_mass_blocks<T>(pb, c, sc));
  // block 3: S^{-1} = Z^{-1} M_gamma Z^{-1} (steady), tau Z~^{-1} (D (x) M_gamma) Z~^{-1} (time)
  if (pb->nt > 1 && pb->opt.schur == 1) {
    SGOC_TRY(coupled_schur<T>(pb, w, r + 2 * F, z + 2 * F, st));
  } else {
    SGOC_TRY(hgs<T>(pb, w, r + 2 * F, w.W1, pb->slabs, st));
    MassArgs<T> m = mass_base<T>(pb, w.W2);
    mass_add(m, w.W1, 0, pb->nt > 0 ? pb->tau : 1.0, pb->nt > 0 ? 3 : 1, ps);
    SGOC_LAUNCH(launch_mass<T>(m, st));
    SGOC_TRY(hgs<T>(pb, w, w.W2, z + 2 * F, pb->slabs, st));
  }
  if (f) SGOC_TRY(fork_to(f->s1, st, f->e[4]));
  return SGOC_OK;
}

// ------------------------------------------------------------------ MINRES --
struct KrylovWS64 {
  double *b, *r, *t, *x;                  // float64 rhs, residual, product, iterate
  double* partial; double* scal; MinresState* state;
};

template <typename T>
struct MinresVecs { T *vp, *v, *z, *zn, *Kz, *wm1, *wm2; };

// Buffer roles of the next iteration: v_{j+1} was written into vp, z_{j+1} into
// zn and w_j into wm2, so the roles swap with period two.
template <typename T>
static MinresVecs<T> swapped(const MinresVecs<T>& m) {
  MinresVecs<T> s = m;
  s.vp = m.v; s.v = m.vp; s.z = m.zn; s.zn = m.z; s.wm1 = m.wm2; s.wm2 = m.wm1;
  return s;
}

template <typename T>
static void carve_minres(const sgoc_problem* pb, Carver& c, MinresVecs<T>& m) {
  const size_t N = size_t(pb->N);
  m.vp = c.template take<T>(N); m.v = c.template take<T>(N); m.z = c.template take<T>(N);
  m.zn = c.template take<T>(N); m.Kz = c.template take<T>(N); m.wm1 = c.template take<T>(N);
  m.wm2 = c.template take<T>(N);
}

// FGMRES workspace: basis V (restart + 1 vectors) and preconditioned vectors Z (restart), each
// of ld entries (ld: N rounded up to 64 entries, so every vector starts 256-byte aligned),
// the Arnoldi vector w, the scalar state and the multi-dot partials.
struct FgWS {
  void* V = nullptr; void* Z = nullptr; void* w = nullptr;
  int64_t ld = 0; int m = 0;
  FgmresState* st = nullptr; double* partial = nullptr;
};

struct Layout {
  FgWS fg;
  KrylovWS64 k64{};
  MinresVecs<double> m64{};
  MinresVecs<float> m32{};
  float* rhs32 = nullptr;   // unit-norm residual of the refinement step
  float* c32 = nullptr;     // inner correction
  PrecWS<double> p64;
  PrecWS<float> p32;
};

static size_t carve_layout(const sgoc_problem* pb, int precision, void* base, size_t cap, Layout& L) {
  Carver c(base, cap, base == nullptr);
  const size_t N = size_t(pb->N);
  L.k64.b = c.take<double>(N);
  L.k64.r = c.take<double>(N);
  L.k64.t = c.take<double>(N);
  L.k64.x = c.take<double>(N);
  L.k64.partial = c.take<double>(kDotBlocks);
  L.k64.scal = c.take<double>(16);
  L.k64.state = c.take<MinresState>(1);
  const bool fg = pb->opt.krylov == 1;
  if (fg) {
    const int m = pb->opt.restart;
    const size_t ld = (N + 63) & ~size_t(63);
    const size_t es = precision == SGOC_FP64 ? 8 : 4;
    L.fg.m = m; L.fg.ld = int64_t(ld);
    L.fg.V = c.take<unsigned char>(es * ld * size_t(m + 1));
    L.fg.Z = c.take<unsigned char>(es * ld * size_t(m));
    L.fg.w = c.take<unsigned char>(es * ld);
    L.fg.st = c.take<FgmresState>(1);
    L.fg.partial = c.take<double>(size_t(kFgmresMax + 1) * kDotBlocks);
  }
  if (precision == SGOC_FP64) {
    if (!fg) carve_minres(pb, c, L.m64);
    carve_prec(pb, c, L.p64);
  } else {
    if (!fg) carve_minres(pb, c, L.m32);
    L.rhs32 = c.take<float>(N);
    L.c32 = c.take<float>(N);
    carve_prec(pb, c, L.p32);
  }
  return c.off;
}

size_t workspace_bytes(const sgoc_problem* pb, int precision) {
  Layout L;
  return carve_layout(pb, precision, nullptr, 0, L);
}

template <typename T> static PrecWS<T>& prec_of(Layout& L);
template <> PrecWS<double>& prec_of<double>(Layout& L) { return L.p64; }
template <> PrecWS<float>& prec_of<float>(Layout& L) { return L.p32; }
template <typename T> static MinresVecs<T>& vecs_of(Layout& L);
template <> MinresVecs<double>& vecs_of<double>(Layout& L) { return L.m64; }
template <> MinresVecs<float>& vecs_of<float>(Layout& L) { return L.m32; }

// Host-side resources of a problem's solves: pinned mirrors of the device
// scalars, a private capture stream and the captured MINRES iteration graphs.
struct Runtime {
  MinresState* hstate = nullptr;
  FgmresState* hfg = nullptr;          // pinned mirror of the FGMRES state header (allocated on first use)
  double* hscal = nullptr;
  cudaStream_t cap = nullptr;
  const void* ws = nullptr;
  int prec = -1;
  cudaGraphExec_t it[2] = {nullptr, nullptr};
  int64_t nk[2] = {0, 0};
  cudaEvent_t ev = nullptr;            // completion of the pending unit of a solve
  Fork fork;                           // auxiliary streams of the parallel branches
  void drop_graphs() {
    for (auto& g : it) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    ws = nullptr; prec = -1;
  }
  ~Runtime() {
    drop_graphs();
    if (cap) cudaStreamDestroy(cap);
    if (ev) cudaEventDestroy(ev);
    if (fork.s1) cudaStreamDestroy(fork.s1);
    if (fork.s2) cudaStreamDestroy(fork.s2);
    if (fork.s3) cudaStreamDestroy(fork.s3);
    for (auto& e : fork.e) if (e) cudaEventDestroy(e);
    if (hstate) cudaFreeHost(hstate);
    if (hfg) cudaFreeHost(hfg);
    if (hscal) cudaFreeHost(hscal);
  }
};

// Parallel branches are left out while per-kernel timing is on: overlapping
// kernels would inflate each other's event-bracketed durations.
static const Fork* fork_of(Runtime* rt) { return profile_enabled() ? nullptr : &rt->fork; }

static void drop_group_graphs(const sgoc_problem* pb);

void invalidate_graphs(sgoc_problem* pb) {
  if (pb->runtime) static_cast<Runtime*>(pb->runtime)->drop_graphs();
  drop_group_graphs(pb);
}

void release_runtime(sgoc_problem* pb) {
  drop_group_graphs(pb);
  delete static_cast<Runtime*>(pb->runtime);
  pb->runtime = nullptr;
}

static sgoc_status runtime_of(sgoc_problem* pb, Runtime** out) {
  if (!pb->runtime) {
    auto* rt = new Runtime();
    pb->runtime = rt;
    SGOC_CUDA_TRY(cudaMallocHost(&rt->hstate, sizeof(MinresState)));
    SGOC_CUDA_TRY(cudaMallocHost(&rt->hscal, 16 * sizeof(double)));
    // the iteration's critical chain is captured on a high-priority stream, its side branches
    // (Chebyshev blocks, deferred w/x update, KKT block rows 2 and 3) on low-priority ones; the
    // graphs keep these priorities, so concurrent solves schedule critical kernels first
    int least = 0, greatest = 0;
    SGOC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    SGOC_CUDA_TRY(cudaStreamCreateWithPriority(&rt->cap, cudaStreamNonBlocking, greatest));
    SGOC_CUDA_TRY(cudaEventCreateWithFlags(&rt->ev, cudaEventDisableTiming));
    SGOC_CUDA_TRY(cudaStreamCreateWithPriority(&rt->fork.s1, cudaStreamNonBlocking, least));
    SGOC_CUDA_TRY(cudaStreamCreateWithPriority(&rt->fork.s2, cudaStreamNonBlocking, least));
    SGOC_CUDA_TRY(cudaStreamCreateWithPriority(&rt->fork.s3, cudaStreamNonBlocking, least));
    for (auto& e : rt->fork.e) SGOC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  *out = static_cast<Runtime*>(pb->runtime);
  return SGOC_OK;
}

// MINRES start: v_1 = rhs, z_1 = P^{-1} v_1, beta_1 = sqrt(v_1 . z_1), w = 0.
template <typename T>
static sgoc_status minres_start(const sgoc_problem* pb, Layout& L, const MinresVecs<T>& m, const T* rhs,
                                double target, cudaStream_t st, const Fork* f) {
  const int64_t N = pb->N;
  SGOC_LAUNCH(launch_scale<T>(rhs, m.v, N, T(1), st));
  SGOC_TRY(precond_apply<T>(pb, prec_of<T>(L), m.v, m.z, st, f));
  SGOC_LAUNCH(launch_dot_partial<T>(m.v, m.z, N, L.k64.partial, st));
  SGOC_LAUNCH(launch_minres_init(L.k64.state, L.k64.partial, target, st));
  SGOC_LAUNCH(launch_fill<T>(m.wm1, N, T(0), st));
  SGOC_LAUNCH(launch_fill<T>(m.wm2, N, T(0), st));
  return SGOC_OK;
}

// The w/x update left pending by the last rotation, with the buffer roles `m` of the
// iteration that follows it (a no-op when nothing is pending).
template <typename T, typename TX>
static sgoc_status prev_wx(const sgoc_problem* pb, Layout& L, const MinresVecs<T>& m, TX* x, cudaStream_t st) {
  SGOC_LAUNCH((launch_minres_wx<T, TX>(m.zn, m.wm2, m.wm1, x, pb->N, L.k64.state, st)));
  return SGOC_OK;
}

// One MINRES iteration with fixed buffer roles (see swapped()).
template <typename T, typename TX>
static sgoc_status minres_step(const sgoc_problem* pb, Layout& L, const MinresVecs<T>& m, TX* x, cudaStream_t st,
                               const Fork* f) {
  const int64_t N = pb->N;
  // The w/x update of the previous iteration j runs here, beside the KKT product: its
  // coefficients stay in the state until this iteration's rotation, and its operands in
  // this iteration's roles are z_j = zn, w_{j-1} = wm2 (read) and w_{j-2} = wm1 (overwritten
  // by w_j).  It joins before the preconditioner, which overwrites zn.  (The update of the
  // last iteration is applied by the caller, prev_wx, when the iteration loop ends.)
  cudaStream_t sw = f ? f->s3 : st;
  if (f) SGOC_TRY(fork_to(st, sw, f->e[6]));
  SGOC_TRY((prev_wx<T, TX>(pb, L, m, x, sw)));
  SGOC_TRY(kkt_apply<T>(pb, m.z, m.Kz, st, f));
  SGOC_LAUNCH(launch_dot_partial<T>(m.z, m.Kz, N, L.k64.partial, st));
  SGOC_LAUNCH(launch_minres_alpha(L.k64.state, L.k64.partial, st));
  // v_{j+1}: its third block row (the multiplier block, all the hGS sweeps read) on the
  // main stream, the first two ahead of the Chebyshev blocks on their branch
  const int64_t F2 = 2 * pb->F;
  SGOC_LAUNCH(launch_minres_v<T>(m.Kz + F2, m.v + F2, m.vp + F2, N - F2, L.k64.state, st));
  if (f) SGOC_TRY(fork_to(sw, st, f->e[7]));
  SGOC_TRY(precond_apply<T>(pb, prec_of<T>(L), m.vp, m.zn, st, f, [&](cudaStream_t sc) -> sgoc_status {
    SGOC_LAUNCH(launch_minres_v<T>(m.Kz, m.v, m.vp, F2, L.k64.state, sc));
    return SGOC_OK;
  }));
  SGOC_LAUNCH(launch_dot_partial<T>(m.vp, m.zn, N, L.k64.partial, st));
  SGOC_LAUNCH(launch_minres_rotate(L.k64.state, L.k64.partial, st));
  return SGOC_OK;
}

// Capture both parities of the iteration (plus the copy of the scalar state to
// the pinned host mirror) into executable graphs, once per workspace.
template <typename T, typename TX>
static sgoc_status ensure_graphs(sgoc_problem* pb, Runtime& rt, Layout& L, const void* ws, TX* x) {
  const int prec = std::is_same<T, double>::value ? 0 : 1;
  if (rt.ws == ws && rt.prec == prec && rt.it[0] && rt.it[1]) return SGOC_OK;
  rt.drop_graphs();
  MinresVecs<T> m = vecs_of<T>(L);
  for (int par = 0; par < 2; ++par) {
    const MinresVecs<T> mp = par == 0 ? m : swapped(m);
    const int64_t k0 = kernel_launches();
    SGOC_CUDA_TRY(cudaStreamBeginCapture(rt.cap, cudaStreamCaptureModeRelaxed));
    sgoc_status s = minres_step<T, TX>(pb, L, mp, x, rt.cap, &rt.fork);
    cudaError_t ce = cudaMemcpyAsync(rt.hstate, L.k64.state, sizeof(MinresState), cudaMemcpyDeviceToHost, rt.cap);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(rt.cap, &g);
    const int64_t nk = kernel_launches() - k0;
    add_launches(-nk);                      // counted when the graph runs
    if (s != SGOC_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_status(ce != cudaSuccess ? ce : ee, "iteration graph capture");
    }
    cudaError_t ie = cudaGraphInstantiateWithFlags(&rt.it[par], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    SGOC_TRY(cuda_status(ie, "cudaGraphInstantiate"));
    rt.nk[par] = nk;
  }
  rt.ws = ws;
  rt.prec = prec;
  return SGOC_OK;
}

// ------------------------------------------------------- group iterations --
// One MINRES iteration of several problems of one shape (sgoc_solve_batch groups
// them): each member's KKT product, inner products, recurrences and Chebyshev
// blocks run on the member's own streams (parallel graph branches), while the two
// hGS sweeps of the Schur blocks run merged over all members (hgs_multi: one SG and
// one V-cycle launch per level visit for the whole group).  Member g uses its own
// buffer roles (parity) and its own scalar state; its arithmetic is that of
// minres_step, so the iterates are bitwise those of the member solved alone.
struct GroupMember {
  sgoc_problem* pb;
  Runtime* rt;
  Layout* L;
  int par;          // buffer roles of this iteration
  void* x;          // the member's iterate (double* or float*)
};

struct GroupRuntime {
  cudaStream_t st = nullptr;                 // launch / capture stream of the group iterations
  cudaEvent_t done = nullptr;                // completion of the group iteration in flight
  std::vector<cudaEvent_t> ev;               // fork / join events (6 per member)
  ~GroupRuntime() {
    if (st) cudaStreamDestroy(st);
    if (done) cudaEventDestroy(done);
    for (auto e : ev) if (e) cudaEventDestroy(e);
  }
  sgoc_status init() {
    int least = 0, greatest = 0;
    SGOC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    SGOC_CUDA_TRY(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest));
    SGOC_CUDA_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    ev.assign(6 * kMaxGroup, nullptr);
    for (auto& e : ev) SGOC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return SGOC_OK;
  }
};

template <typename T, typename TX>
static sgoc_status group_step(const std::vector<GroupMember>& gm, GroupRuntime& gr, bool copy_state) {
  const int ng = int(gm.size());
  cudaStream_t gs = gr.st;
  std::vector<MinresVecs<T>> mv(ng);
  std::vector<HgsMember<T>> h1(ng), h2(ng);
  for (int g = 0; g < ng; ++g) {
    const GroupMember& m = gm[g];
    const MinresVecs<T>& base = vecs_of<T>(*m.L);
    mv[g] = m.par == 0 ? base : swapped(base);
    PrecWS<T>& w = prec_of<T>(*m.L);
    h1[g] = HgsMember<T>{m.pb, &w, mv[g].vp + 2 * m.pb->F, w.W1};
    h2[g] = HgsMember<T>{m.pb, &w, w.W2, mv[g].zn + 2 * m.pb->F};
  }
  // A: per member, everything the first hGS sweep waits for (and the Chebyshev branch)
  for (int g = 0; g < ng; ++g) {
    const GroupMember& m = gm[g];
    const sgoc_problem* pb = m.pb;
    Layout& L = *m.L;
    const MinresVecs<T>& v = mv[g];
    TX* x = static_cast<TX*>(m.x);
    const Fork* f = fork_of(m.rt);
    cudaStream_t cs = m.rt->cap;
    SGOC_TRY(fork_to(gs, cs, gr.ev[6 * g + 0]));
    const int64_t N = pb->N, F2 = 2 * pb->F;
    cudaStream_t sw = f ? f->s3 : cs;
    if (f) SGOC_TRY(fork_to(cs, sw, f->e[6]));
    SGOC_TRY((prev_wx<T, TX>(pb, L, v, x, sw)));
    SGOC_TRY(kkt_apply<T>(pb, v.z, v.Kz, cs, f));
    SGOC_LAUNCH(launch_dot_partial<T>(v.z, v.Kz, N, L.k64.partial, cs));
    SGOC_LAUNCH(launch_minres_alpha(L.k64.state, L.k64.partial, cs));
    SGOC_LAUNCH(launch_minres_v<T>(v.Kz + F2, v.v + F2, v.vp + F2, N - F2, L.k64.state, cs));
    if (f) SGOC_TRY(fork_to(sw, cs, f->e[7]));
    // Chebyshev blocks 1, 2 of the preconditioner on their branch (as in precond_apply)
    PrecWS<T>& w = prec_of<T>(L);
    ChebArgs<T> c{};
    c.B = v.vp; c.X = v.zn; c.tmpA = w.chebA; c.tmpB = w.chebB;
    c.ncols = 2 * int64_t(pb->slabs) * pb->P; c.n1 = pb->n1; c.n = pb->n; c.steps = pb->opt.cheb_steps;
    c.mass = T(pb->mass_h2_36); c.scale_mode = 1; c.P = pb->P; c.slabs = pb->slabs; c.nt = pb->nt;
    c.tau = T(pb->tau); c.beta = T(pb->beta); c.gamma = T(pb->gamma);
    cudaStream_t sc = cs;
    if (f) { SGOC_TRY(fork_to(cs, f->s1, f->e[3])); sc = f->s1; }
    SGOC_LAUNCH(launch_minres_v<T>(v.Kz, v.v, v.vp, F2, L.k64.state, sc));
    SGOC_LAUNCH(launch_mass_blocks<T>(pb, c, sc));
    SGOC_TRY(fork_to(cs, gs, gr.ev[6 * g + 1]));
  }
  // B: the first hGS sweep of every member, merged
  SGOC_TRY(hgs_multi<T>(h1, gm[0].pb->slabs, gs));
  // C: per member, W2 = M_gamma W1 (steady) or tau (D (x) M_gamma) W1 (time)
  for (int g = 0; g < ng; ++g) {
    const sgoc_problem* pb = gm[g].pb;
    cudaStream_t cs = gm[g].rt->cap;
    PrecWS<T>& w = prec_of<T>(*gm[g].L);
    SGOC_TRY(fork_to(gs, cs, gr.ev[6 * g + 2]));
    MassArgs<T> ma = mass_base<T>(pb, w.W2);
    mass_add(ma, w.W1, 0, pb->nt > 0 ? pb->tau : 1.0, pb->nt > 0 ? 3 : 1, int64_t(pb->P) * pb->n);
    SGOC_LAUNCH(launch_mass<T>(ma, cs));
    SGOC_TRY(fork_to(cs, gs, gr.ev[6 * g + 3]));
  }
  // D: the second hGS sweep, merged
  SGOC_TRY(hgs_multi<T>(h2, gm[0].pb->slabs, gs));
  // E: per member, the Chebyshev branch joins, then v.z and the rotation
  for (int g = 0; g < ng; ++g) {
    const GroupMember& m = gm[g];
    const sgoc_problem* pb = m.pb;
    Layout& L = *m.L;
    const Fork* f = fork_of(m.rt);
    cudaStream_t cs = m.rt->cap;
    SGOC_TRY(fork_to(gs, cs, gr.ev[6 * g + 4]));
    if (f) SGOC_TRY(fork_to(f->s1, cs, f->e[4]));
    SGOC_LAUNCH(launch_dot_partial<T>(mv[g].vp, mv[g].zn, pb->N, L.k64.partial, cs));
    SGOC_LAUNCH(launch_minres_rotate(L.k64.state, L.k64.partial, cs));
    if (copy_state) {
      SGOC_CUDA_TRY(cudaMemcpyAsync(m.rt->hstate, L.k64.state, sizeof(MinresState), cudaMemcpyDeviceToHost, cs));
      pdl_fence(cs);
    }
    SGOC_TRY(fork_to(cs, gs, gr.ev[6 * g + 5]));
  }
  return SGOC_OK;
}

// Captured group iterations, keyed by the members (problem, workspace, buffer roles) in
// order; a graph refers to device addresses of its members' problem data and
// workspaces, so it is dropped when any member is re-uploaded or destroyed.
struct GroupGraph { cudaGraphExec_t exec = nullptr; int64_t nk = 0; };
using GroupKey = std::vector<std::tuple<const void*, const void*, int>>;
static std::mutex g_group_mu;
static std::map<GroupKey, GroupGraph> g_group_graphs;

static void drop_group_graphs(const sgoc_problem* pb) {
  std::lock_guard<std::mutex> lk(g_group_mu);
  for (auto it = g_group_graphs.begin(); it != g_group_graphs.end();) {
    bool hit = false;
    for (const auto& t : it->first) hit = hit || std::get<0>(t) == pb;
    if (hit) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      it = g_group_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

// Enqueue one iteration of the group on gr.st (a captured graph, or eagerly while
// per-kernel timing is on) and record gr.done.
template <typename T, typename TX>
static sgoc_status launch_group_iteration(const std::vector<GroupMember>& gm, const std::vector<const void*>& ws,
                                          GroupRuntime& gr, bool graphs) {
  for (const auto& m : gm) SGOC_CUDA_TRY(cudaStreamWaitEvent(gr.st, m.rt->ev, 0));   // each member's last unit
  pdl_fence(gr.st);
  if (!graphs) {
    SGOC_TRY((group_step<T, TX>(gm, gr, true)));
    pdl_fence(gr.st);
    SGOC_CUDA_TRY(cudaEventRecord(gr.done, gr.st));
    return SGOC_OK;
  }
  GroupKey key;
  for (size_t g = 0; g < gm.size(); ++g) key.emplace_back(gm[g].pb, ws[g], gm[g].par);
  GroupGraph gg;
  {
    std::lock_guard<std::mutex> lk(g_group_mu);
    auto it = g_group_graphs.find(key);
    if (it != g_group_graphs.end()) gg = it->second;
  }
  if (!gg.exec) {
    const int64_t k0 = kernel_launches();
    SGOC_CUDA_TRY(cudaStreamBeginCapture(gr.st, cudaStreamCaptureModeRelaxed));
    sgoc_status s = group_step<T, TX>(gm, gr, true);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(gr.st, &g);
    gg.nk = kernel_launches() - k0;
    add_launches(-gg.nk);                       // counted when the graph runs
    if (s != SGOC_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (ee != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_status(ee, "group iteration capture"); }
    cudaError_t ie = cudaGraphInstantiateWithFlags(&gg.exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    SGOC_TRY(cuda_status(ie, "cudaGraphInstantiate (group)"));
    std::lock_guard<std::mutex> lk(g_group_mu);
    g_group_graphs[key] = gg;
  }
  SGOC_CUDA_TRY(cudaGraphLaunch(gg.exec, gr.st));
  add_launches(gg.nk);
  pdl_fence(gr.st);
  SGOC_CUDA_TRY(cudaEventRecord(gr.done, gr.st));
  return SGOC_OK;
}

static sgoc_status state_error(const MinresState& hs) {
  if (hs.flag == 4) { set_error("NaN in MINRES recurrences"); return SGOC_ERR_NAN; }
  if (hs.flag == 3) { set_error("preconditioner not positive definite"); return SGOC_ERR_NOT_SPD; }
  return SGOC_OK;
}

static sgoc_status rhs_apply(const sgoc_problem* pb, double* b, cudaStream_t st) {
  SGOC_LAUNCH(launch_fill<double>(b, pb->N, 0.0, st));
  MassArgs<double> m = mass_base<double>(pb, b);
  m.ncols = 1;
  // block 1, chaos column 0: M yhat (steady) or tau D_t M yhat_t (time)
  mass_add(m, pb->dev.yhat, 0, pb->nt > 0 ? pb->tau : 1.0, pb->nt > 0 ? 2 : 0, pb->n);
  SGOC_LAUNCH(launch_mass<double>(m, st));
  if (pb->nt > 0 && !pb->y0.empty()) {
    // block 3: -d with d = [M y0 e_1, 0, ...]
    MassArgs<double> m3 = mass_base<double>(pb, b + 2 * pb->F);
    m3.ncols = 1; m3.nslabs = 1;
    mass_add(m3, pb->dev.y0, 0, -1.0, 0, pb->n);
    SGOC_LAUNCH(launch_mass<double>(m3, st));
  }
  return SGOC_OK;
}

static sgoc_status check_ready(const sgoc_problem* pb) {
  if (!pb) { set_error("null problem"); return SGOC_ERR_INVALID_ARG; }
  if (!pb->uploaded) { set_error("call sgoc_problem_upload first"); return SGOC_ERR_NOT_UPLOADED; }
  return SGOC_OK;
}

static sgoc_status check_ws(void* ws, size_t bytes, size_t need) {
  if (bytes < need) { set_error("workspace too small: need " + std::to_string(need)); return SGOC_ERR_WORKSPACE_TOO_SMALL; }
  if (need && !ws) { set_error("null workspace"); return SGOC_ERR_INVALID_ARG; }
  if (reinterpret_cast<uintptr_t>(ws) % 256) { set_error("workspace must be 256-byte aligned"); return SGOC_ERR_INVALID_ARG; }
  return SGOC_OK;
}

// A solve in progress, as a resumable state machine.  begin() enqueues the first
// unit of device work; every unit ends by copying the scalars the host needs
// (norms or the MINRES state) to pinned host memory and recording `ev`.  After
// `ev` has completed, step() reads those scalars, takes the decision of the
// stopping rule and enqueues the next unit.  One host thread can thus keep many
// solves in flight on their own streams (sgoc_solve_batch, the server).
struct SolveTask {
  enum Phase { BNORM, R0, START64, ITER64, CHECK64, OUTER, START32, ITER32, FSTART64, FITER64, FCHECK64,
               FSTART32, FITER32, DONE };
  sgoc_problem* pb = nullptr;
  Runtime* rt = nullptr;
  Layout L;
  cudaStream_t st = nullptr;
  void* ws = nullptr;
  const double* x0 = nullptr;
  double* x_out = nullptr;
  bool graphs = true;
  // grouped: the iterations of this solve run inside its group's merged iterations
  // (sgoc_solve_batch): launch_iter only marks the solve as waiting for the next one
  bool grouped = false, want_iter = false, in_group = false;
  Phase phase = DONE;
  double bnorm = 0, target = 0, rn = 0;
  int j = 0, jin = 0, par = 0, outer = 0, total = 0, last_flag = 0;
  int fj = 0;                          // FGMRES: columns of the current cycle
  bool fgmres() const { return pb->opt.krylov == 1; }
  sgoc_status status = SGOC_OK;
  sgoc_result result{};
  std::chrono::steady_clock::time_point t0;

  sgoc_status record() { SGOC_CUDA_TRY(cudaEventRecord(rt->ev, st)); return SGOC_OK; }

  sgoc_status launch_norm(const double* a) {
    SGOC_LAUNCH(launch_dot_partial<double>(a, a, pb->N, L.k64.partial, st));
    SGOC_LAUNCH(launch_sum_partials(L.k64.partial, L.k64.scal, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(rt->hscal, L.k64.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    pdl_fence(st);
    return record();
  }
  sgoc_status launch_true_residual() {
    SGOC_TRY(kkt_apply<double>(pb, L.k64.x, L.k64.t, st, fork_of(rt)));
    SGOC_LAUNCH(launch_sub(L.k64.b, L.k64.t, L.k64.r, pb->N, st));
    return launch_norm(L.k64.r);
  }
  template <typename T, typename TX>
  sgoc_status launch_start(const T* rhs, double tgt) {
    SGOC_TRY(minres_start<T>(pb, L, vecs_of<T>(L), rhs, tgt, st, fork_of(rt)));
    SGOC_CUDA_TRY(cudaMemcpyAsync(rt->hstate, L.k64.state, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
    pdl_fence(st);
    par = 0;
    return record();
  }
  template <typename T, typename TX>
  sgoc_status launch_iter(TX* x) {
    if (grouped) { want_iter = true; return SGOC_OK; }
    if (graphs) {
      SGOC_CUDA_TRY(cudaGraphLaunch(rt->it[par], st));
      pdl_fence(st);
      add_launches(rt->nk[par]);
    } else {
      const MinresVecs<T>& m = vecs_of<T>(L);
      SGOC_TRY((minres_step<T, TX>(pb, L, par == 0 ? m : swapped(m), x, st, fork_of(rt))));
      SGOC_CUDA_TRY(cudaMemcpyAsync(rt->hstate, L.k64.state, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
      pdl_fence(st);
    }
    par ^= 1;
    return record();
  }
  // apply the pending w/x update of the last iteration (roles of the next parity) and clear it
  template <typename T, typename TX>
  sgoc_status flush_wx(TX* x) {
    const MinresVecs<T>& m = vecs_of<T>(L);
    SGOC_TRY((prev_wx<T, TX>(pb, L, par == 0 ? m : swapped(m), x, st)));
    SGOC_CUDA_TRY(cudaMemsetAsync(&L.k64.state->wx_pending, 0, sizeof(int), st));
    pdl_fence(st);
    return SGOC_OK;
  }
  // ---- FGMRES units (Sec. 5): one Arnoldi step per unit, the host reads the state header ----
  sgoc_status fg_head() {
    SGOC_CUDA_TRY(cudaMemcpyAsync(rt->hfg, L.fg.st, offsetof(FgmresState, h), cudaMemcpyDeviceToHost, st));
    pdl_fence(st);
    return record();
  }
  // a cycle from rhs (the residual of the current iterate): v_0 = rhs / ||rhs||
  template <typename T>
  sgoc_status fg_start(const T* rhs, double tgt, double bn) {
    if (!rt->hfg) SGOC_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&rt->hfg), offsetof(FgmresState, h)));
    SGOC_LAUNCH(launch_dot_partial<T>(rhs, rhs, pb->N, L.k64.partial, st));
    SGOC_LAUNCH(launch_fgmres_start(L.fg.st, L.k64.partial, tgt, bn, st));
    SGOC_LAUNCH(launch_fgmres_scale<T>(rhs, static_cast<T*>(L.fg.V), pb->N, L.fg.st, 0, st));
    fj = 0;
    return fg_head();
  }
  // z_j = P^{-1} v_j, w = K z_j, two classical Gram-Schmidt passes, h_{j+1,j} = ||w||,
  // rotations and estimate, v_{j+1} = w / h_{j+1,j}
  template <typename T>
  sgoc_status fg_iter() {
    T* V = static_cast<T*>(L.fg.V);
    T* Z = static_cast<T*>(L.fg.Z);
    T* w = static_cast<T*>(L.fg.w);
    const int64_t ld = L.fg.ld, N = pb->N;
    SGOC_TRY(precond_apply<T>(pb, prec_of<T>(L), V + fj * ld, Z + fj * ld, st, fork_of(rt)));
    SGOC_TRY(kkt_apply<T>(pb, Z + fj * ld, w, st, fork_of(rt)));
    for (int pass = 0; pass < 2; ++pass) {
      SGOC_LAUNCH(launch_fgmres_multidot<T>(V, ld, w, N, L.fg.st, pass, L.fg.partial, st));
      SGOC_LAUNCH((launch_fgmres_axpy<T, T>(w, V, ld, N, L.fg.st, pass, st)));
    }
    SGOC_LAUNCH(launch_dot_partial<T>(w, w, N, L.k64.partial, st));
    SGOC_LAUNCH(launch_fgmres_rotate(L.fg.st, L.k64.partial, st));
    SGOC_LAUNCH(launch_fgmres_scale<T>(w, V + (fj + 1) * ld, N, L.fg.st, 1, st));
    return fg_head();
  }
  // x += Z y for the cycle's columns (enqueued; the caller's next unit follows)
  template <typename T, typename TX>
  sgoc_status fg_end(TX* x) {
    SGOC_LAUNCH(launch_fgmres_solve_y(L.fg.st, st));
    SGOC_LAUNCH((launch_fgmres_axpy<T, TX>(x, static_cast<const T*>(L.fg.Z), L.fg.ld, pb->N, L.fg.st, 2, st)));
    return SGOC_OK;
  }
  sgoc_status fg_state_error(const FgmresState& h) {
    if (h.flag == 4) { set_error("NaN in FGMRES recurrences"); return SGOC_ERR_NAN; }
    return SGOC_OK;
  }

  sgoc_status finish(sgoc_status s) {
    status = s;
    phase = DONE;
    cudaError_t e = cudaMemcpyAsync(x_out, L.k64.x, pb->N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    pdl_fence(st);
    if (status == SGOC_OK && e != cudaSuccess) status = cuda_status(e, "copy solution");
    if (status == SGOC_OK && pb->opt.mean_solve != 0) {
      bool failed = false;
      e = spectral_take_error(&failed, st);
      if (e != cudaSuccess) status = cuda_status(e, "exact mean solve status");
      else if (failed) { set_error("exact mean solve: a bounded wait on the tensor cores ran out"); status = SGOC_ERR_CUDA; }
    }
    result.status = status;
    return status;
  }
  sgoc_status fail(sgoc_status s) {
    status = s;
    phase = DONE;
    result.status = s;
    return s;
  }

  sgoc_status begin(sgoc_problem* p, void* d_ws, size_t ws_bytes, const double* d_x0, double* d_x, cudaStream_t s) {
    t0 = std::chrono::steady_clock::now();
    pb = p; ws = d_ws; x0 = d_x0; x_out = d_x; st = s;
    pdl_fence(st);                                 // the caller's prior work on st
    result = sgoc_result{};
    status = SGOC_OK;
    bnorm = target = rn = 0;
    j = jin = par = outer = total = last_flag = 0;
    carve_layout(pb, pb->opt.precision, d_ws, ws_bytes, L);
    SGOC_TRY(runtime_of(pb, &rt));
    graphs = !profile_enabled();
    if (graphs && !fgmres()) {
      if (pb->opt.precision == SGOC_FP64) SGOC_TRY((ensure_graphs<double, double>(pb, *rt, L, ws, L.k64.x)));
      else SGOC_TRY((ensure_graphs<float, float>(pb, *rt, L, ws, L.c32)));
    }
    SGOC_TRY(rhs_apply(pb, L.k64.b, st));
    phase = BNORM;
    return launch_norm(L.k64.b);
  }

  // Consume the completed unit and enqueue the next one.
  sgoc_status step() {
    const double tol = pb->opt.tol;
    const int64_t N = pb->N;
    switch (phase) {
      case BNORM: {
        bnorm = std::sqrt(rt->hscal[0]);
        if (bnorm == 0.0) { SGOC_LAUNCH(launch_fill<double>(L.k64.x, N, 0.0, st)); return finish(SGOC_OK); }
        if (!std::isfinite(bnorm)) { set_error("non-finite right-hand side"); return fail(SGOC_ERR_NAN); }
        if (x0) {
          SGOC_CUDA_TRY(cudaMemcpyAsync(L.k64.x, x0, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
          pdl_fence(st);
        } else {
          SGOC_LAUNCH(launch_fill<double>(L.k64.x, N, 0.0, st));
        }
        if (pb->opt.precision != SGOC_FP64) { phase = OUTER; return launch_true_residual(); }
        if (x0) { phase = R0; return launch_true_residual(); }
        target = tol;
        if (fgmres()) { phase = FSTART64; return fg_start<double>(L.k64.b, target, bnorm); }
        phase = START64;
        return launch_start<double, double>(L.k64.b, target);
      }
      case R0: {
        // the stopping rule is relative to b: with an initial guess the estimate target
        // is rescaled by ||b|| / ||r0|| (2-norms) and the true residual decides at exit
        const double rn0 = std::sqrt(rt->hscal[0]);
        result.rel_true_residual = rn0 / bnorm;
        if (rn0 / bnorm <= tol) return finish(SGOC_OK);
        if (fgmres()) {                              // estimates are relative to ||b||: target tol
          target = tol;
          phase = FSTART64;
          return fg_start<double>(L.k64.r, target, bnorm);
        }
        target = std::min(0.5, tol * bnorm / rn0);
        phase = START64;
        return launch_start<double, double>(L.k64.r, target);
      }
      case START64:
      case START32: {
        sgoc_status e = state_error(*rt->hstate);
        if (e != SGOC_OK) return fail(e);
        jin = 0;
        phase = phase == START64 ? ITER64 : ITER32;
        if (phase == ITER64) return launch_iter<double, double>(L.k64.x);
        return launch_iter<float, float>(L.c32);
      }
      case ITER64: {
        const MinresState hs = *rt->hstate;
        ++j;
        result.iterations = j; result.outer_iterations = 1; result.rel_estimate = hs.est;
        sgoc_status e = state_error(hs);
        if (e != SGOC_OK) return fail(e);
        if (hs.flag == 1 || hs.flag == 2 || j >= pb->opt.max_iter) SGOC_TRY((flush_wx<double, double>(L.k64.x)));
        if (hs.flag == 1 || hs.flag == 2) { last_flag = hs.flag; phase = CHECK64; return launch_true_residual(); }
        if (j >= pb->opt.max_iter) { set_error("MINRES iteration limit reached"); return finish(SGOC_ERR_NO_CONVERGENCE); }
        return launch_iter<double, double>(L.k64.x);
      }
      case CHECK64: {
        const double rel = std::sqrt(rt->hscal[0]) / bnorm;
        result.rel_true_residual = rel;
        if (rel <= tol || last_flag == 2) return finish(SGOC_OK);
        if (j >= pb->opt.max_iter) { set_error("MINRES iteration limit reached"); return finish(SGOC_ERR_NO_CONVERGENCE); }
        target *= tol / rel;
        rt->hstate->target = target;
        rt->hstate->flag = 0;
        SGOC_CUDA_TRY(cudaMemcpyAsync(&L.k64.state->target, &rt->hstate->target, sizeof(double),
                                      cudaMemcpyHostToDevice, st));
        SGOC_CUDA_TRY(cudaMemcpyAsync(&L.k64.state->flag, &rt->hstate->flag, sizeof(int), cudaMemcpyHostToDevice, st));
        pdl_fence(st);
        phase = ITER64;
        return launch_iter<double, double>(L.k64.x);
      }
      case OUTER: {
        rn = std::sqrt(rt->hscal[0]);
        const double rel = rn / bnorm;
        result.rel_true_residual = rel; result.outer_iterations = outer; result.iterations = total;
        if (!std::isfinite(rel)) { set_error("non-finite residual in refinement"); return fail(SGOC_ERR_NAN); }
        if (rel <= tol) return finish(SGOC_OK);
        if (outer >= pb->opt.max_outer) { set_error("iterative refinement step limit reached"); return finish(SGOC_ERR_NO_CONVERGENCE); }
        // unit-norm residual in float32, inner solve K c = r / ||r||, then x += ||r|| c
        SGOC_LAUNCH(launch_scale_to32(L.k64.r, L.rhs32, N, 1.0 / rn, st));
        SGOC_LAUNCH(launch_fill<float>(L.c32, N, 0.0f, st));
        if (fgmres()) { jin = 0; phase = FSTART32; return fg_start<float>(L.rhs32, pb->opt.inner_tol, 1.0); }
        phase = START32;
        return launch_start<float, float>(L.rhs32, pb->opt.inner_tol);
      }
      case ITER32: {
        const MinresState hs = *rt->hstate;
        ++jin; ++total;
        result.rel_estimate = hs.est; result.iterations = total;
        sgoc_status e = state_error(hs);
        if (e != SGOC_OK) return fail(e);
        if (hs.flag == 1 || hs.flag == 2 || jin >= pb->opt.max_iter) {
          SGOC_TRY((flush_wx<float, float>(L.c32)));
          SGOC_LAUNCH(launch_add_scaled(L.c32, L.k64.x, N, rn, st));
          ++outer;
          phase = OUTER;
          return launch_true_residual();
        }
        return launch_iter<float, float>(L.c32);
      }
      case FSTART64:
      case FSTART32: {
        sgoc_status e = fg_state_error(*rt->hfg);
        if (e != SGOC_OK) return fail(e);
        phase = phase == FSTART64 ? FITER64 : FITER32;
        if (phase == FITER64) return fg_iter<double>();
        return fg_iter<float>();
      }
      case FITER64: {
        const FgmresState hs = *rt->hfg;
        ++j;
        result.iterations = j; result.outer_iterations = 1; result.rel_estimate = hs.est;
        sgoc_status e = fg_state_error(hs);
        if (e != SGOC_OK) return fail(e);
        fj = hs.j;
        if (hs.flag == 0 && fj < L.fg.m && j < pb->opt.max_iter) return fg_iter<double>();
        last_flag = hs.flag;
        SGOC_TRY((fg_end<double, double>(L.k64.x)));
        phase = FCHECK64;
        return launch_true_residual();
      }
      case FCHECK64: {
        const double rel = std::sqrt(rt->hscal[0]) / bnorm;
        result.rel_true_residual = rel;
        if (rel <= tol) return finish(SGOC_OK);
        if (j >= pb->opt.max_iter) { set_error("FGMRES iteration limit reached"); return finish(SGOC_ERR_NO_CONVERGENCE); }
        if (last_flag == 1) target *= tol / rel;       // the estimate fired early: tighten it
        phase = FSTART64;                             // restart from the current iterate
        return fg_start<double>(L.k64.r, target, bnorm);
      }
      case FITER32: {
        const FgmresState hs = *rt->hfg;
        ++jin; ++total;
        result.rel_estimate = hs.est; result.iterations = total;
        sgoc_status e = fg_state_error(hs);
        if (e != SGOC_OK) return fail(e);
        fj = hs.j;
        if (hs.flag == 0 && fj < L.fg.m && jin < pb->opt.max_iter) return fg_iter<float>();
        SGOC_TRY((fg_end<float, float>(L.c32)));
        SGOC_LAUNCH(launch_add_scaled(L.c32, L.k64.x, N, rn, st));
        ++outer;
        phase = OUTER;
        return launch_true_residual();
      }
      case DONE:
        return status;
    }
    return status;
  }

  // wait for the pending unit (host blocks) and advance
  sgoc_status wait_and_step() {
    cudaError_t e = cudaEventSynchronize(rt->ev);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaEventSynchronize"));
    sgoc_status s = step();
    if (s != SGOC_OK && phase != DONE) return fail(s);
    return s;
  }
};

// ----------------------------------------------------------------- server --
// First-fit sub-allocator over the caller's device pool (offsets, 256-B aligned).
class PoolAllocator {
 public:
  explicit PoolAllocator(size_t bytes) { free_[0] = bytes; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct ServerRequest {
  sgoc_problem* pb;
  double* d_x;
  uint64_t id;
  std::chrono::steady_clock::time_point t_submit;
};

struct ServerSlot {
  bool busy = false;
  cudaStream_t st = nullptr;
  SolveTask task;
  ServerRequest req{};
  size_t off = 0, bytes = 0, pers = 0;
  std::chrono::steady_clock::time_point t_admit;
};

}  // namespace sgoc

struct sgoc_server {
  char* pool = nullptr;
  size_t pool_bytes = 0;
  sgoc::PoolAllocator alloc{0};
  std::vector<sgoc::ServerSlot> slots;
  std::deque<sgoc::ServerRequest> queue;
  std::vector<std::pair<uint64_t, sgoc_result>> done;
  int64_t admitted = 0, completed = 0, rejected = 0;
  size_t high_water = 0;
};

namespace sgoc {

static sgoc_status server_admit(sgoc_server* sv) {
  while (!sv->queue.empty()) {
    ServerSlot* slot = nullptr;
    for (auto& s : sv->slots) if (!s.busy) { slot = &s; break; }
    if (!slot) return SGOC_OK;
    ServerRequest& rq = sv->queue.front();
    const size_t pers = align256(rq.pb->persistent_bytes);
    const size_t need = pers + workspace_bytes(rq.pb, rq.pb->opt.precision);
    size_t off = 0;
    if (!sv->alloc.alloc(need, &off)) return SGOC_OK;     // FIFO: wait for memory
    slot->busy = true;
    slot->req = rq;
    slot->off = off; slot->bytes = need; slot->pers = pers;
    slot->t_admit = std::chrono::steady_clock::now();
    sv->queue.pop_front();
    sv->admitted++;
    sv->high_water = std::max(sv->high_water, sv->alloc.used());
    char* base = sv->pool + off;
    sgoc_status s = sgoc_problem_upload(slot->req.pb, base, pers, slot->st);
    if (s == SGOC_OK) s = slot->task.begin(slot->req.pb, base + pers, need - pers, nullptr, slot->req.d_x, slot->st);
    if (s != SGOC_OK) slot->task.fail(s);
  }
  return SGOC_OK;
}

static void server_retire(sgoc_server* sv, ServerSlot& slot) {
  cudaStreamSynchronize(slot.st);
  sgoc_result r = slot.task.result;
  r.status = slot.task.status;
  r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - slot.req.t_submit).count();
  sv->done.emplace_back(slot.req.id, r);
  sv->alloc.release(slot.off, slot.bytes);
  slot.req.pb->uploaded = false;           // its device data lived in the pool
  slot.busy = false;
  sv->completed++;
}

}  // namespace sgoc

extern "C" {

sgoc_status sgoc_server_create(void* d_pool, size_t pool_bytes, int32_t max_active, sgoc_server** out) {
  using namespace sgoc;
  if (!out || !d_pool || pool_bytes < 256 || max_active < 1 || max_active > 1024 ||
      reinterpret_cast<uintptr_t>(d_pool) % 256) {
    set_error("server: pool must be non-null, >= 256 bytes and 256-byte aligned; 1 <= max_active <= 1024");
    return SGOC_ERR_INVALID_ARG;
  }
  auto* sv = new sgoc_server();
  sv->pool = static_cast<char*>(d_pool);
  sv->pool_bytes = pool_bytes;
  sv->alloc = PoolAllocator(pool_bytes);
  sv->slots.resize(max_active);
  for (auto& s : sv->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { sgoc_server_destroy(sv); return cuda_status(e, "server stream"); }
  }
  *out = sv;
  return SGOC_OK;
}

void sgoc_server_destroy(sgoc_server* sv) {
  if (!sv) return;
  for (auto& s : sv->slots) {
    if (s.st) { cudaStreamSynchronize(s.st); cudaStreamDestroy(s.st); }
    if (s.busy) s.req.pb->uploaded = false;
  }
  delete sv;
}

sgoc_status sgoc_server_submit(sgoc_server* sv, sgoc_problem* pb, double* d_x, uint64_t request_id) {
  using namespace sgoc;
  if (!sv || !pb || !d_x) { set_error("server submit: null argument"); return SGOC_ERR_INVALID_ARG; }
  const size_t need = align256(pb->persistent_bytes) + workspace_bytes(pb, pb->opt.precision);
  if (need > sv->pool_bytes) {
    sv->rejected++;
    set_error("server submit: request needs " + std::to_string(need) + " bytes, more than the whole pool");
    return SGOC_ERR_WORKSPACE_TOO_SMALL;
  }
  sv->queue.push_back(ServerRequest{pb, d_x, request_id, std::chrono::steady_clock::now()});
  return SGOC_OK;
}

sgoc_status sgoc_server_step(sgoc_server* sv, int32_t* n_active, int32_t* n_queued) {
  using namespace sgoc;
  if (!sv) { set_error("null server"); return SGOC_ERR_INVALID_ARG; }
  SGOC_TRY(server_admit(sv));
  // advance every active solve whose pending unit has completed; if none has,
  // block on the oldest one so that the sweep always makes progress
  bool progressed = false;
  ServerSlot* oldest = nullptr;
  for (auto& s : sv->slots) {
    if (!s.busy) continue;
    if (s.task.phase == SolveTask::DONE) { server_retire(sv, s); progressed = true; continue; }
    if (!oldest || s.t_admit < oldest->t_admit) oldest = &s;
    if (cudaEventQuery(s.task.rt->ev) == cudaSuccess) {
      s.task.wait_and_step();
      progressed = true;
      if (s.task.phase == SolveTask::DONE) server_retire(sv, s);
    }
  }
  if (!progressed && oldest) {
    oldest->task.wait_and_step();
    if (oldest->task.phase == SolveTask::DONE) server_retire(sv, *oldest);
  }
  SGOC_TRY(server_admit(sv));
  int act = 0;
  for (auto& s : sv->slots) act += s.busy ? 1 : 0;
  if (n_active) *n_active = act;
  if (n_queued) *n_queued = int32_t(sv->queue.size());
  return SGOC_OK;
}

sgoc_status sgoc_server_poll(sgoc_server* sv, uint64_t* ids, sgoc_result* res, int32_t cap, int32_t* n_done) {
  using namespace sgoc;
  if (!sv || !n_done || cap < 0 || (cap > 0 && (!ids || !res))) { set_error("server poll: bad arguments"); return SGOC_ERR_INVALID_ARG; }
  const int n = std::min<int>(cap, int(sv->done.size()));
  for (int i = 0; i < n; ++i) { ids[i] = sv->done[i].first; res[i] = sv->done[i].second; }
  sv->done.erase(sv->done.begin(), sv->done.begin() + n);
  *n_done = n;
  return SGOC_OK;
}

sgoc_status sgoc_server_stats(const sgoc_server* sv, int64_t* admitted, int64_t* completed, int64_t* rejected,
                              size_t* pool_high_water) {
  using namespace sgoc;
  if (!sv) { set_error("null server"); return SGOC_ERR_INVALID_ARG; }
  if (admitted) *admitted = sv->admitted;
  if (completed) *completed = sv->completed;
  if (rejected) *rejected = sv->rejected;
  if (pool_high_water) *pool_high_water = sv->high_water;
  return SGOC_OK;
}

}  // extern "C"

namespace sgoc {

template <typename T>
static sgoc_status prec_hook(sgoc_problem* pb, void* ws, size_t bytes, PrecWS<T>& w) {
  const size_t need = precond_workspace_bytes(pb, sizeof(T));
  SGOC_TRY(check_ws(ws, bytes, need));
  Carver c(ws, bytes, false);
  carve_prec(pb, c, w);
  return SGOC_OK;
}

}  // namespace sgoc

using namespace sgoc;


// SG launch shape `shape` of a solve (0 KKT product, 1 operator alone, 2 + d return visit of hGS
// level d, 3 + p + d first visit of level d)
// with placeholder pointers: the tuning table is keyed by the shape only.
template <typename T>
static bool shape_args(sgoc_problem* pb, int shape, SGArgs<T>* out) {
  static T dummy[1];
  if (shape == 0 || shape == 1) {
    SGArgs<T> g = sg_full<T>(pb, dummy, dummy, T(shape == 0 ? -1 : 1));
    if (shape == 1) g.cy = T(0);
    if (!g.u_mb) g.u_mb = reinterpret_cast<const int*>(dummy);       // slot table exists once uploaded
    *out = g;
    return true;
  }
  const int d = shape - 2 <= pb->p ? shape - 2 : shape - 3 - pb->p;
  if (shape < 2 || d < 0 || d > pb->p) return false;
  PrecWS<T> w;
  w.RH = dummy;
  *out = shape - 2 <= pb->p ? hgs_args<T>(pb, w, dummy, dummy, pb->slabs, d)
                            : hgs_args_first<T>(pb, w, dummy, dummy, pb->slabs, d);
  if (!out->u_mb) out->u_mb = reinterpret_cast<const int*>(dummy);   // slot table exists once uploaded
  return true;
}

// ------------------------------------------------------------------ tuning --
// Times every feasible SG kernel variant on each SG launch shape of a solve of
// this problem (the KKT product, the operator alone, each hGS level visit) on the
// caller's workspace and records the fastest in the tuning cache.
template <typename T>
static sgoc_status tune_sg_shape(const SGArgs<T>& a, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps,
                                 double* best_ms, int* best_v) {
  *best_v = -1;
  *best_ms = 1e30;
  // each variant: two warm-up launches, then the best of three rounds of `reps` launches (one
  // round alone was seen to pick a twice slower kernel now and then)
  for (int v = 0; v < kSGVariants; ++v) {
    if (!sg_variant_feasible(a, v)) continue;
    for (int w = 0; w < 2; ++w) SGOC_LAUNCH(launch_sg_variant<T>(a, v, st));
    double best_round = 1e30;
    for (int round = 0; round < 3; ++round) {
      SGOC_CUDA_TRY(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) SGOC_LAUNCH(launch_sg_variant<T>(a, v, st));
      SGOC_CUDA_TRY(cudaEventRecord(e1, st));
      SGOC_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0;
      SGOC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      best_round = std::min(best_round, double(ms) / reps);
    }
    if (best_round < *best_ms) { *best_ms = best_round; *best_v = v; }
  }
  if (*best_v >= 0) sg_set_variant(a, *best_v);
  return SGOC_OK;
}

template <typename T>
static sgoc_status tune_problem(sgoc_problem* pb, Layout& L, PrecWS<T>& w, T* X, T* Y, cudaStream_t st,
                                cudaEvent_t e0, cudaEvent_t e1, int32_t* chosen, int nchosen) {
  const int64_t F = pb->F;
  SGOC_LAUNCH(launch_fill<T>(X, F, T(0), st));
  SGOC_LAUNCH(launch_fill<T>(Y, F, T(0), st));
  SGOC_LAUNCH(launch_fill<T>(w.RH, int64_t(pb->slabs) * level_columns_max(pb) * pb->n, T(0), st));
  std::vector<SGArgs<T>> shapes;
  shapes.push_back(sg_full<T>(pb, X, Y, T(-1)));               // KKT product rows (accumulating)
  SGArgs<T> op = sg_full<T>(pb, X, Y, T(1));
  op.cy = T(0);
  shapes.push_back(op);                                       // the operator alone
  for (int d = 0; d <= pb->p; ++d) shapes.push_back(hgs_args<T>(pb, w, Y, X, pb->slabs, d));
  for (int d = 0; d <= pb->p; ++d) shapes.push_back(hgs_args_first<T>(pb, w, Y, X, pb->slabs, d));
  int k = 0;
  for (const SGArgs<T>& a : shapes) {
    double ms = 0;
    int v = -1;
    SGOC_TRY(tune_sg_shape<T>(a, st, e0, e1, 5, &ms, &v));
    if (chosen && k < nchosen) chosen[k] = v;
    ++k;
  }
  (void)L;
  return SGOC_OK;
}

extern "C" {

int64_t sgoc_kernel_launches(void) { return kernel_launches(); }

sgoc_status sgoc_profile_enable(int32_t on) {
  profile_enable(on != 0);
  return SGOC_OK;
}

sgoc_status sgoc_profile_query(int32_t kind, int64_t* launches, double* ms, double* bytes, double* flops) {
  if (kind < 0 || kind >= KK_COUNT || !launches || !ms || !bytes || !flops) {
    set_error("bad kernel kind or null output");
    return SGOC_ERR_INVALID_ARG;
  }
  if (!profile_query(kind, launches, ms, bytes, flops)) {
    set_error("event query failed");
    return SGOC_ERR_CUDA;
  }
  return SGOC_OK;
}

const char* sgoc_kernel_kind_name(int32_t kind) { return kernel_kind_name(kind); }

sgoc_status sgoc_inner_product(int32_t precision, const void* d_a, const void* d_b, int64_t n, void* d_ws,
                               size_t ws_bytes, double* d_out, void* stream) {
  static_assert(SGOC_INNER_PRODUCT_WS_BYTES >= kDotBlocks * sizeof(double), "inner-product scratch too small");
  if ((n > 0 && (!d_a || !d_b)) || !d_out || !d_ws || n < 0 || (precision != 0 && precision != 1)) {
    set_error("inner product: null pointer, negative length or bad precision");
    return SGOC_ERR_INVALID_ARG;
  }
  if (ws_bytes < SGOC_INNER_PRODUCT_WS_BYTES || reinterpret_cast<uintptr_t>(d_ws) % 8) {
    set_error("inner product: scratch must hold SGOC_INNER_PRODUCT_WS_BYTES bytes, 8-byte aligned");
    return SGOC_ERR_WORKSPACE_TOO_SMALL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  double* partial = static_cast<double*>(d_ws);
  if (precision == 0) SGOC_LAUNCH(launch_dot_partial<double>(static_cast<const double*>(d_a),
                                                             static_cast<const double*>(d_b), n, partial, st));
  else SGOC_LAUNCH(launch_dot_partial<float>(static_cast<const float*>(d_a), static_cast<const float*>(d_b), n,
                                             partial, st));
  SGOC_LAUNCH(launch_sum_partials(partial, d_out, st));
  return SGOC_OK;
}

sgoc_status sgoc_rhs(sgoc_problem* pb, double* d_b, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_b) { set_error("null output"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  return rhs_apply(pb, d_b, st);
}

sgoc_status sgoc_solve(sgoc_problem* pb, void* d_ws, size_t ws_bytes, const double* d_x0, double* d_x,
                       void* stream, sgoc_result* res) {
  SGOC_TRY(check_ready(pb));
  if (!d_x) { set_error("null solution buffer"); return SGOC_ERR_INVALID_ARG; }
  SGOC_TRY(check_ws(d_ws, ws_bytes, workspace_bytes(pb, pb->opt.precision)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  SolveTask task;
  sgoc_status s = task.begin(pb, d_ws, ws_bytes, d_x0, d_x, st);
  if (s != SGOC_OK) task.fail(s);
  while (task.phase != SolveTask::DONE) task.wait_and_step();
  s = task.status;
  cudaError_t e = cudaStreamSynchronize(st);
  if (s == SGOC_OK && e != cudaSuccess) s = cuda_status(e, "cudaStreamSynchronize");
  if (res) {
    *res = task.result;
    res->status = s;
    res->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - task.t0).count();
  }
  return s;
}

static sgoc_status solve_batch_impl(int32_t count, sgoc_problem* const* pbs, void* const* d_ws,
                                   const size_t* ws_bytes, const double* const* d_x0, double* const* d_x,
                                   void* const* streams, sgoc_result* res, bool merge) {
  if (count < 0 || (count > 0 && (!pbs || !d_ws || !ws_bytes || !d_x || !streams))) {
    set_error("bad batch arguments");
    return SGOC_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    SGOC_TRY(check_ready(pbs[i]));
    if (!d_x[i]) { set_error("null solution buffer"); return SGOC_ERR_INVALID_ARG; }
    SGOC_TRY(check_ws(d_ws[i], ws_bytes[i], workspace_bytes(pbs[i], pbs[i]->opt.precision)));
    for (int k = 0; k < i; ++k)
      if (pbs[k] == pbs[i]) { set_error("a problem may appear only once in a batch"); return SGOC_ERR_INVALID_ARG; }
  }
  std::vector<SolveTask> tasks(count);
  for (int i = 0; i < count; ++i) {
    sgoc_status s = tasks[i].begin(pbs[i], d_ws[i], ws_bytes[i], d_x0 ? d_x0[i] : nullptr, d_x[i],
                                   static_cast<cudaStream_t>(streams[i]));
    if (s != SGOC_OK) tasks[i].fail(s);
  }
  // merged schedule: problems of one shape whose mean solves can run merged form groups;
  // their MINRES iterations run together (group_step), each level visit of the hGS
  // sweeps as one SG and one mean-solve launch (V-cycle or exact) for the whole group
  struct Group { GroupRuntime gr; std::vector<int> members, active; bool inflight = false; };
  std::vector<std::unique_ptr<Group>> groups;
  if (merge) {
    std::vector<std::vector<int>> cand;
    for (int i = 0; i < count; ++i) {
      if (tasks[i].phase == SolveTask::DONE || pbs[i]->opt.krylov != 0) continue;   // MINRES iterations only
      const int esize = pbs[i]->opt.precision == SGOC_FP64 ? 8 : 4;
      const VPlan vp = plan_vcycle(pbs[i], esize);
      if (vp.lf != 0 || vp.cluster) continue;
      bool placed = false;
      for (auto& c : cand)
        if (int(c.size()) < kMaxGroup && same_shape(pbs[c[0]], pbs[i])) { c.push_back(i); placed = true; break; }
      if (!placed) cand.push_back({i});
    }
    for (auto& c : cand) {
      if (c.size() < 2) continue;
      auto g = std::make_unique<Group>();
      sgoc_status s = g->gr.init();
      if (s != SGOC_OK) return s;
      g->members = c;
      for (int i : c) tasks[i].grouped = true;
      groups.push_back(std::move(g));
    }
  }
  auto group_launch = [&](Group& G) -> sgoc_status {
    std::vector<GroupMember> gm;
    std::vector<const void*> ws;
    for (int i : G.active) {
      SolveTask& t = tasks[i];
      const bool f64 = t.pb->opt.precision == SGOC_FP64;
      gm.push_back(GroupMember{t.pb, t.rt, &t.L, t.par, f64 ? static_cast<void*>(t.L.k64.x) : static_cast<void*>(t.L.c32)});
      ws.push_back(t.ws);
    }
    const bool f64 = tasks[G.active[0]].pb->opt.precision == SGOC_FP64;
    const bool graphs = tasks[G.active[0]].graphs;
    if (f64) return launch_group_iteration<double, double>(gm, ws, G.gr, graphs);
    return launch_group_iteration<float, float>(gm, ws, G.gr, graphs);
  };
  // advance each solve as soon as its pending unit has completed (polling, so that no solve
  // waits behind another); yield the host thread while none is ready
  for (bool busy = true; busy;) {
    busy = false;
    bool progressed = false;
    for (auto& t : tasks) {
      if (t.phase == SolveTask::DONE) continue;
      busy = true;
      if (t.want_iter || t.in_group) continue;
      const cudaError_t q = cudaEventQuery(t.rt->ev);
      if (q != cudaErrorNotReady) {               // completed, or an error wait_and_step reports
        t.wait_and_step();
        progressed = true;
      }
    }
    for (auto& gp : groups) {
      Group& G = *gp;
      if (G.inflight) {
        const cudaError_t q = cudaEventQuery(G.gr.done);
        if (q == cudaErrorNotReady) continue;
        G.inflight = false;
        progressed = true;
        for (int i : G.active) {
          SolveTask& t = tasks[i];
          t.in_group = false;
          if (q != cudaSuccess) { t.fail(cuda_status(q, "group iteration")); continue; }
          // the solve's next units on its own stream follow the group iteration
          cudaError_t we = cudaStreamWaitEvent(t.st, G.gr.done, 0);
          if (we != cudaSuccess) { t.fail(cuda_status(we, "cudaStreamWaitEvent")); continue; }
          pdl_fence(t.st);
          sgoc_status s = t.step();
          if (s != SGOC_OK && t.phase != SolveTask::DONE) t.fail(s);
        }
      }
      if (!G.inflight) {
        G.active.clear();
        for (int i : G.members)
          if (tasks[i].phase != SolveTask::DONE && tasks[i].want_iter) G.active.push_back(i);
        if (G.active.empty()) continue;
        sgoc_status s = group_launch(G);
        for (int i : G.active) {
          SolveTask& t = tasks[i];
          t.want_iter = false;
          if (s != SGOC_OK) { t.fail(s); continue; }
          t.in_group = true;
          t.par ^= 1;
        }
        G.inflight = s == SGOC_OK;
        progressed = true;
      }
    }
    if (busy && !progressed) std::this_thread::yield();
  }
  sgoc_status first = SGOC_OK;
  for (int i = 0; i < count; ++i) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(streams[i]));
    sgoc_status s = tasks[i].status;
    if (s == SGOC_OK && e != cudaSuccess) s = cuda_status(e, "cudaStreamSynchronize");
    if (res) {
      res[i] = tasks[i].result;
      res[i].status = s;
      res[i].ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tasks[i].t0).count();
    }
    if (first == SGOC_OK) first = s;
  }
  return first;
}

sgoc_status sgoc_solve_batch(int32_t count, sgoc_problem* const* pbs, void* const* d_ws, const size_t* ws_bytes,
                             const double* const* d_x0, double* const* d_x, void* const* streams,
                             sgoc_result* res) {
  return solve_batch_impl(count, pbs, d_ws, ws_bytes, d_x0, d_x, streams, res, false);
}

sgoc_status sgoc_solve_batch_merged(int32_t count, sgoc_problem* const* pbs, void* const* d_ws,
                                    const size_t* ws_bytes, const double* const* d_x0, double* const* d_x,
                                    void* const* streams, sgoc_result* res) {
  return solve_batch_impl(count, pbs, d_ws, ws_bytes, d_x0, d_x, streams, res, true);
}

sgoc_status sgoc_apply_operator(sgoc_problem* pb, int32_t precision, const void* d_X, void* d_Y, int32_t nslabs,
                                void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_X || !d_Y || nslabs < 1) { set_error("bad arguments"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) {
    SGArgs<double> g = sg_full<double>(pb, static_cast<const double*>(d_X), static_cast<double*>(d_Y), 1.0);
    g.cy = 0.0; g.nslabs = nslabs;
    return cuda_status(launch_sg<double>(g, st), "sg apply");
  }
  if (precision == 1) {
    SGArgs<float> g = sg_full<float>(pb, static_cast<const float*>(d_X), static_cast<float*>(d_Y), 1.0f);
    g.cy = 0.0f; g.nslabs = nslabs;
    return cuda_status(launch_sg<float>(g, st), "sg apply");
  }
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}

sgoc_status sgoc_apply_kkt(sgoc_problem* pb, int32_t precision, const void* d_v, void* d_w, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_v || !d_w) { set_error("bad arguments"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) return kkt_apply<double>(pb, static_cast<const double*>(d_v), static_cast<double*>(d_w), st);
  if (precision == 1) return kkt_apply<float>(pb, static_cast<const float*>(d_v), static_cast<float*>(d_w), st);
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}

sgoc_status sgoc_apply_precond(sgoc_problem* pb, int32_t precision, const void* d_r, void* d_z, void* d_ws,
                               size_t ws_bytes, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_r || !d_z) { set_error("bad arguments"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) {
    PrecWS<double> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    return precond_apply<double>(pb, w, static_cast<const double*>(d_r), static_cast<double*>(d_z), st);
  }
  if (precision == 1) {
    PrecWS<float> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    return precond_apply<float>(pb, w, static_cast<const float*>(d_r), static_cast<float*>(d_z), st);
  }
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}

sgoc_status sgoc_apply_hgs(sgoc_problem* pb, int32_t precision, const void* d_R, void* d_V, int32_t nslabs,
                           void* d_ws, size_t ws_bytes, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_R || !d_V || nslabs < 1 || nslabs > pb->slabs) { set_error("bad arguments"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) {
    PrecWS<double> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    return hgs<double>(pb, w, static_cast<const double*>(d_R), static_cast<double*>(d_V), nslabs, st);
  }
  if (precision == 1) {
    PrecWS<float> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    return hgs<float>(pb, w, static_cast<const float*>(d_R), static_cast<float*>(d_V), nslabs, st);
  }
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}

sgoc_status sgoc_apply_vcycle(sgoc_problem* pb, int32_t precision, const void* d_R, void* d_X, int32_t ncols,
                              void* d_ws, size_t ws_bytes, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_R || !d_X || ncols < 1 || ncols > pb->slabs * level_columns_max(pb)) {
    set_error("bad arguments (ncols must not exceed slabs * largest level size)");
    return SGOC_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) {
    PrecWS<double> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    return vcycle<double>(pb, w, static_cast<const double*>(d_R), static_cast<double*>(d_X), ncols, nullptr, 0, 1, 0, st);
  }
  if (precision == 1) {
    PrecWS<float> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    return vcycle<float>(pb, w, static_cast<const float*>(d_R), static_cast<float*>(d_X), ncols, nullptr, 0, 1, 0, st);
  }
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}

sgoc_status sgoc_apply_chebyshev(sgoc_problem* pb, int32_t precision, const void* d_R, void* d_X, int32_t ncols,
                                 void* d_ws, size_t ws_bytes, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_R || !d_X || ncols < 1 || int64_t(ncols) > 2 * int64_t(pb->slabs) * pb->P) {
    set_error("bad arguments (ncols must not exceed 2 * slabs * P)");
    return SGOC_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) {
    PrecWS<double> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    ChebArgs<double> c{};
    c.B = static_cast<const double*>(d_R); c.X = static_cast<double*>(d_X); c.tmpA = w.chebA; c.tmpB = w.chebB;
    c.ncols = ncols; c.n1 = pb->n1; c.n = pb->n; c.steps = pb->opt.cheb_steps; c.mass = pb->mass_h2_36;
    c.scale_mode = 0;
    return cuda_status(launch_cheb<double>(c, st), "chebyshev");
  }
  if (precision == 1) {
    PrecWS<float> w; SGOC_TRY(prec_hook(pb, d_ws, ws_bytes, w));
    ChebArgs<float> c{};
    c.B = static_cast<const float*>(d_R); c.X = static_cast<float*>(d_X); c.tmpA = w.chebA; c.tmpB = w.chebB;
    c.ncols = ncols; c.n1 = pb->n1; c.n = pb->n; c.steps = pb->opt.cheb_steps; c.mass = float(pb->mass_h2_36);
    c.scale_mode = 0;
    return cuda_status(launch_cheb<float>(c, st), "chebyshev");
  }
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}


sgoc_status sgoc_autotune(sgoc_problem* pb, void* d_ws, size_t ws_bytes, int32_t* chosen, int32_t nchosen,
                          void* stream) {
  SGOC_TRY(check_ready(pb));
  SGOC_TRY(check_ws(d_ws, ws_bytes, workspace_bytes(pb, pb->opt.precision)));
  if (nchosen < 0 || (nchosen > 0 && !chosen)) { set_error("bad chosen array"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  Layout L;
  carve_layout(pb, pb->opt.precision, d_ws, ws_bytes, L);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SGOC_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_status(ce, "cudaEventCreate"); }
  sgoc_status s;
  if (pb->opt.precision == SGOC_FP64) {
    s = tune_problem<double>(pb, L, L.p64, L.k64.r, L.k64.t, st, e0, e1, chosen, nchosen);
  } else {
    // float32 shapes on the mixed workspace, then the float64 true-residual product
    s = tune_problem<float>(pb, L, L.p32, L.rhs32, L.c32, st, e0, e1, chosen, nchosen);
    if (s == SGOC_OK) {
      double ms = 0;
      int v = -1;
      s = tune_sg_shape<double>(sg_full<double>(pb, L.k64.r, L.k64.t, -1.0), st, e0, e1, 3, &ms, &v);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  invalidate_graphs(pb);          // captured iterations carry the kernels chosen before
  return s;
}


sgoc_status sgoc_apply_operator_variant(sgoc_problem* pb, int32_t precision, int32_t variant, const void* d_X,
                                        void* d_Y, int32_t nslabs, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_X || !d_Y || nslabs < 1 || variant < 0 || variant >= kSGVariants) {
    set_error("bad arguments");
    return SGOC_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) {
    SGArgs<double> g = sg_full<double>(pb, static_cast<const double*>(d_X), static_cast<double*>(d_Y), 1.0);
    g.cy = 0.0; g.nslabs = nslabs;
    if (!sg_variant_feasible(g, variant)) { set_error("kernel variant not applicable"); return SGOC_ERR_UNSUPPORTED; }
    return cuda_status(launch_sg_variant<double>(g, variant, st), "sg apply");
  }
  if (precision == 1) {
    SGArgs<float> g = sg_full<float>(pb, static_cast<const float*>(d_X), static_cast<float*>(d_Y), 1.0f);
    g.cy = 0.f; g.nslabs = nslabs;
    if (!sg_variant_feasible(g, variant)) { set_error("kernel variant not applicable"); return SGOC_ERR_UNSUPPORTED; }
    return cuda_status(launch_sg_variant<float>(g, variant, st), "sg apply");
  }
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}


sgoc_status sgoc_set_kernel(sgoc_problem* pb, int32_t precision, int32_t shape, int32_t variant) {
  if (!pb) { set_error("null problem"); return SGOC_ERR_INVALID_ARG; }
  if (variant < -1 || variant >= kSGVariants) { set_error("kernel variant out of range"); return SGOC_ERR_INVALID_ARG; }
  if (precision == 0) {
    SGArgs<double> g{};
    if (!shape_args<double>(pb, shape, &g)) { set_error("shape out of range"); return SGOC_ERR_INVALID_ARG; }
    if (variant < 0) { sg_clear_variant(g); return SGOC_OK; }
    if (!sg_variant_feasible(g, variant)) { set_error("kernel variant not applicable"); return SGOC_ERR_UNSUPPORTED; }
    sg_set_variant(g, variant);
  } else if (precision == 1) {
    SGArgs<float> g{};
    if (!shape_args<float>(pb, shape, &g)) { set_error("shape out of range"); return SGOC_ERR_INVALID_ARG; }
    if (variant < 0) { sg_clear_variant(g); return SGOC_OK; }
    if (!sg_variant_feasible(g, variant)) { set_error("kernel variant not applicable"); return SGOC_ERR_UNSUPPORTED; }
    sg_set_variant(g, variant);
  } else {
    set_error("precision must be 0 or 1");
    return SGOC_ERR_INVALID_ARG;
  }
  invalidate_graphs(pb);
  return SGOC_OK;
}

}  // extern "C"
