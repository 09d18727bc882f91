// Solver orchestration: KKT products, block preconditioner (Chebyshev mass
// blocks, hierarchical Gauss-Seidel Schur block with batched V-cycles),
// preconditioned MINRES, float32/float64 iterative refinement and the ABI hooks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
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

// Largest finest level handled by the fused one-CTA-per-column V-cycle.
static int fused_n1_limit(int esize) {
  const int lim = fused_vcycle_max_n1(esize);
  // float64 runs at a small fraction of the float32 rate on this GPU: keep
  // one-SM-per-column work small there and use grid-wide level kernels above.
  return esize == 8 ? (lim < 15 ? lim : 15) : lim;
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
  const int lim = fused_n1_limit(sizeof(T));
  for (int l = 0; l < nl; ++l) {
    const size_t nlv = size_t(pb->levels[l].n);
    w.lx[l] = c.template take<T>(B * nlv);
    if (pb->levels[l].n1 > lim) w.lt[l] = c.template take<T>(B * nlv);
    if (l > 0) w.lb[l] = c.template take<T>(B * nlv);
    if (pb->levels[l].n1 <= lim) break;
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
template <typename T>
static sgoc_status vcycle(const sgoc_problem* pb, PrecWS<T>& w, const T* b, T* xout, int64_t B, T* acc,
                          int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st) {
  const int nl = int(pb->levels.size());
  const int lim = fused_n1_limit(sizeof(T));
  const T om = T(pb->opt.omega);
  const int nu = pb->opt.nu_pre;
  int lf = 0;
  while (lf < nl - 1 && pb->levels[lf].n1 > lim) ++lf;
  FusedLevels FL;
  FL.nlev = nl - lf;
  for (int l = lf; l < nl; ++l) {
    FL.n1[l - lf] = pb->levels[l].n1;
    FL.diag[l - lf] = pb->levels[l].diag; FL.edge[l - lf] = pb->levels[l].edge; FL.corner[l - lf] = pb->levels[l].corner;
  }
  if (lf == 0) {
    SGOC_LAUNCH(launch_vcycle_fused<T>(b, xout, B, FL, om, nu, acc, acc_ss, acc_L, acc_col0, st));
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
  SGOC_LAUNCH(launch_vcycle_fused<T>(bl[lf], w.lx[lf], B, FL, om, nu, (T*)nullptr, 0, 1, 0, st));
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
template <typename T>
static sgoc_status hgs(const sgoc_problem* pb, PrecWS<T>& w, const T* R, T* V, int slabs, cudaStream_t st) {
  const int P = pb->P, p = pb->p;
  const int64_t n = pb->n, ps = int64_t(P) * n;
  SGOC_LAUNCH(launch_fill<T>(V, slabs * ps, T(0), st));
  const bool time = pb->nt > 0;
  const T cK = T(time ? pb->tau : 1.0);                 // multiplies K_0 .. K_M
  const T cM = T(time ? 1.0 + pb->tau * pb->s : pb->s); // multiplies M in the mean operator
  std::vector<int> order;
  for (int d = 0; d <= p; ++d) order.push_back(d);
  for (int d = p - 1; d >= 0; --d) order.push_back(d);
  for (int d : order) {
    const int a0 = pb->off[d], a1 = pb->off[d + 1], L = a1 - a0;
    SGArgs<T> g{};
    g.X = V; g.xs = ps;
    g.Y = w.RH; g.ys = int64_t(L) * n; g.ycol0 = a0;
    g.R = R; g.rs = ps; g.rcol0 = 0;
    g.n1 = pb->n1; g.n = n; g.nx = pb->nx; g.M = pb->M;
    g.out0 = a0; g.out1 = a1;
    g.in0 = pb->off[d > 0 ? d - 1 : 0];
    g.in1 = pb->off[d + 2 <= p + 1 ? d + 2 : p + 1];
    g.kmax = pb->r; g.nslabs = slabs;
    g.c0 = -cK; g.c1 = -cK; g.cm = -cM; g.cr = T(1); g.cy = T(0);
    g.mass = T(pb->mass_h2_36);
    g.kap = kap_of<T>(pb);
    g.nbr_ptr = pb->dev.nbr_ptr; g.nbr_alpha = pb->dev.nbr_alpha; g.nbr_k = pb->dev.nbr_k; g.nbr_c = nbrc_of<T>(pb);
    g.deg_sum = deg_sum(pb, a0, a1, pb->r);
    SGOC_LAUNCH(launch_sg<T>(g, st));
    SGOC_TRY(vcycle<T>(pb, w, w.RH, nullptr, int64_t(slabs) * L, V, ps, L, a0, st));
  }
  return SGOC_OK;
}

// -------------------------------------------------------------- KKT apply --
template <typename T>
static SGArgs<T> sg_full(const sgoc_problem* pb, const T* X, T* Y, T coef) {
  SGArgs<T> g{};
  const int64_t ps = int64_t(pb->P) * pb->n;
  g.X = X; g.xs = ps; g.Y = Y; g.ys = ps; g.ycol0 = 0;
  g.R = nullptr; g.rs = 0; g.rcol0 = 0;
  g.n1 = pb->n1; g.n = pb->n; g.nx = pb->nx; g.M = pb->M;
  g.out0 = 0; g.out1 = pb->P; g.in0 = 0; g.in1 = pb->P;
  g.kmax = pb->M + 1; g.nslabs = pb->slabs;
  g.c0 = coef; g.c1 = coef; g.cm = T(0); g.cr = T(0); g.cy = T(1);
  g.mass = T(pb->mass_h2_36);
  g.kap = kap_of<T>(pb);
  g.nbr_ptr = pb->dev.nbr_ptr; g.nbr_alpha = pb->dev.nbr_alpha; g.nbr_k = pb->dev.nbr_k; g.nbr_c = nbrc_of<T>(pb);
  g.deg_sum = double(pb->nbr_alpha.size());
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
static sgoc_status kkt_apply(const sgoc_problem* pb, const T* v, T* w, cudaStream_t st) {
  const int64_t F = pb->F, ps = int64_t(pb->P) * pb->n;
  const T* y = v; const T* u = v + F; const T* lam = v + 2 * F;
  T* w1 = w; T* w2 = w + F; T* w3 = w + 2 * F;
  if (pb->nt == 0) {
    // w1 = M Y H^gamma - A Lambda ; w2 = beta M U + M Lambda ; w3 = -A Y + M U   (Eq. (stoch-system))
    MassArgs<T> m1 = mass_base<T>(pb, w1); mass_add(m1, y, 0, 1.0, 1, ps);
    SGOC_LAUNCH(launch_mass<T>(m1, st));
    SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, lam, w1, T(-1)), st));
    MassArgs<T> m2 = mass_base<T>(pb, w2); mass_add(m2, u, 0, pb->beta, 0, ps); mass_add(m2, lam, 0, 1.0, 0, ps);
    SGOC_LAUNCH(launch_mass<T>(m2, st));
    MassArgs<T> m3 = mass_base<T>(pb, w3); mass_add(m3, u, 0, 1.0, 0, ps);
    SGOC_LAUNCH(launch_mass<T>(m3, st));
    SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, y, w3, T(-1)), st));
    return SGOC_OK;
  }
  // time (Eq. (KKT:stoch-time-dependent)), A_t = I (x) (M_cal + tau A) - C (x) M_cal:
  // w1_t = tau D_t M Y_t H^g - (M L_t + tau A L_t - M L_{t+1})
  // w2_t = beta tau D_t M U_t + tau M L_t
  // w3_t = -(M Y_t + tau A Y_t - M Y_{t-1}) + tau M U_t
  const double tau = pb->tau;
  MassArgs<T> m1 = mass_base<T>(pb, w1);
  mass_add(m1, y, 0, tau, 3, ps); mass_add(m1, lam, 0, -1.0, 0, ps); mass_add(m1, lam, 1, 1.0, 0, ps);
  SGOC_LAUNCH(launch_mass<T>(m1, st));
  SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, lam, w1, T(-tau)), st));
  MassArgs<T> m2 = mass_base<T>(pb, w2);
  mass_add(m2, u, 0, pb->beta * tau, 2, ps); mass_add(m2, lam, 0, tau, 0, ps);
  SGOC_LAUNCH(launch_mass<T>(m2, st));
  MassArgs<T> m3 = mass_base<T>(pb, w3);
  mass_add(m3, y, 0, -1.0, 0, ps); mass_add(m3, y, -1, 1.0, 0, ps); mass_add(m3, u, 0, tau, 0, ps);
  SGOC_LAUNCH(launch_mass<T>(m3, st));
  SGOC_LAUNCH(launch_sg<T>(sg_full<T>(pb, y, w3, T(-tau)), st));
  return SGOC_OK;
}

// ------------------------------------------------------ block preconditioner --
template <typename T>
static sgoc_status precond_apply(const sgoc_problem* pb, PrecWS<T>& w, const T* r, T* z, cudaStream_t st) {
  const int64_t F = pb->F, ps = int64_t(pb->P) * pb->n;
  // blocks 1, 2: Chebyshev on M, scaled by 1/(sc_t H^gamma) and 1/(sc_t beta)
  ChebArgs<T> c{};
  c.B = r; c.X = z; c.tmpA = w.chebA; c.tmpB = w.chebB;
  c.ncols = 2 * int64_t(pb->slabs) * pb->P; c.n1 = pb->n1; c.n = pb->n; c.steps = pb->opt.cheb_steps;
  c.mass = T(pb->mass_h2_36); c.scale_mode = 1; c.P = pb->P; c.slabs = pb->slabs; c.nt = pb->nt;
  c.tau = T(pb->tau); c.beta = T(pb->beta); c.gamma = T(pb->gamma);
  SGOC_LAUNCH(launch_cheb<T>(c, st));
  // block 3: S^{-1} = Z^{-1} M_gamma Z^{-1} (steady), tau Z~^{-1} (D (x) M_gamma) Z~^{-1} (time)
  SGOC_TRY(hgs<T>(pb, w, r + 2 * F, w.W1, pb->slabs, st));
  MassArgs<T> m = mass_base<T>(pb, w.W2);
  mass_add(m, w.W1, 0, pb->nt > 0 ? pb->tau : 1.0, pb->nt > 0 ? 3 : 1, ps);
  SGOC_LAUNCH(launch_mass<T>(m, st));
  SGOC_TRY(hgs<T>(pb, w, w.W2, z + 2 * F, pb->slabs, st));
  return SGOC_OK;
}

// ------------------------------------------------------------------ MINRES --
struct KrylovWS64 {
  double *b, *r, *t;                      // float64 rhs, residual, product
  double* partial; double* scal; MinresState* state;
};

template <typename T>
struct MinresVecs { T *vp, *v, *z, *zn, *Kz, *wm1, *wm2; };

template <typename T>
static void carve_minres(const sgoc_problem* pb, Carver& c, MinresVecs<T>& m) {
  const size_t N = size_t(pb->N);
  m.vp = c.template take<T>(N); m.v = c.template take<T>(N); m.z = c.template take<T>(N);
  m.zn = c.template take<T>(N); m.Kz = c.template take<T>(N); m.wm1 = c.template take<T>(N);
  m.wm2 = c.template take<T>(N);
}

struct Layout {
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
  L.k64.partial = c.take<double>(kDotBlocks);
  L.k64.scal = c.take<double>(16);
  L.k64.state = c.take<MinresState>(1);
  if (precision == SGOC_FP64) {
    carve_minres(pb, c, L.m64);
    carve_prec(pb, c, L.p64);
  } else {
    carve_minres(pb, c, L.m32);
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

static sgoc_status read_state(const MinresState* d, MinresState* h, cudaStream_t st) {
  SGOC_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
  SGOC_CUDA_TRY(cudaStreamSynchronize(st));
  return SGOC_OK;
}

static sgoc_status norm2(const double* a, int64_t n, double* partial, double* scal_dev, double* out,
                         cudaStream_t st) {
  SGOC_LAUNCH(launch_dot_partial<double>(a, a, n, partial, st));
  SGOC_LAUNCH(launch_sum_partials(partial, scal_dev, st));
  double h = 0;
  SGOC_CUDA_TRY(cudaMemcpyAsync(&h, scal_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  SGOC_CUDA_TRY(cudaStreamSynchronize(st));
  *out = std::sqrt(h);
  return SGOC_OK;
}

// Preconditioned MINRES on K d = rhs (vectors of type T, float64 scalars); the
// iterate accumulates into x.  Stopping: estimate <= target; when `check` is set
// the true float64 residual ||b64 - K x||/||b64|| decides (rule of the oracle).
template <typename T>
static sgoc_status minres(const sgoc_problem* pb, Layout& L, MinresVecs<T>& m, const T* rhs, T* x,
                          double tol, int max_iter, bool check_true, double bnorm, cudaStream_t st,
                          int* iters, double* est_out, double* rel_out) {
  const int64_t N = pb->N;
  PrecWS<T>& pw = prec_of<T>(L);
  MinresState hs{};
  double target = tol;
  *iters = 0;
  // v_1 = rhs, z_1 = P^{-1} v_1
  SGOC_LAUNCH(launch_scale<T>(rhs, m.v, N, T(1), st));
  SGOC_TRY(precond_apply<T>(pb, pw, m.v, m.z, st));
  SGOC_LAUNCH(launch_dot_partial<T>(m.v, m.z, N, L.k64.partial, st));
  SGOC_LAUNCH(launch_minres_init(L.k64.state, L.k64.partial, target, st));
  SGOC_LAUNCH(launch_fill<T>(m.wm1, N, T(0), st));
  SGOC_LAUNCH(launch_fill<T>(m.wm2, N, T(0), st));
  SGOC_TRY(read_state(L.k64.state, &hs, st));
  if (hs.flag == 3) { set_error("<v, P^-1 v> <= 0 at start"); return SGOC_ERR_NOT_SPD; }
  if (hs.flag == 4) { set_error("NaN at start"); return SGOC_ERR_NAN; }
  double rel = 1.0;
  for (int j = 1; j <= max_iter; ++j) {
    SGOC_TRY(kkt_apply<T>(pb, m.z, m.Kz, st));
    SGOC_LAUNCH(launch_dot_partial<T>(m.z, m.Kz, N, L.k64.partial, st));
    SGOC_LAUNCH(launch_minres_alpha(L.k64.state, L.k64.partial, st));
    SGOC_LAUNCH(launch_minres_v<T>(m.Kz, m.v, m.vp, N, L.k64.state, st));   // vp <- v_{j+1}
    SGOC_TRY(precond_apply<T>(pb, pw, m.vp, m.zn, st));
    SGOC_LAUNCH(launch_dot_partial<T>(m.vp, m.zn, N, L.k64.partial, st));
    SGOC_LAUNCH(launch_minres_rotate(L.k64.state, L.k64.partial, st));
    SGOC_LAUNCH(launch_minres_wx<T, T>(m.z, m.wm1, m.wm2, x, N, L.k64.state, st));  // wm2 <- w_j
    std::swap(m.vp, m.v);     // v <- v_{j+1}, vp <- v_j
    std::swap(m.z, m.zn);
    std::swap(m.wm1, m.wm2);  // wm1 <- w_j, wm2 <- w_{j-1}
    SGOC_TRY(read_state(L.k64.state, &hs, st));
    *iters = j;
    *est_out = hs.est;
    if (hs.flag == 4) { set_error("NaN in MINRES recurrences"); return SGOC_ERR_NAN; }
    if (hs.flag == 3) { set_error("preconditioner not positive definite"); return SGOC_ERR_NOT_SPD; }
    if (hs.flag == 1 || hs.flag == 2) {
      if (!check_true) return SGOC_OK;
      // true float64 residual of the outer system (only used with float64 iterates)
      double rn = 0;
      if constexpr (std::is_same<T, double>::value) {
        SGOC_TRY(kkt_apply<double>(pb, x, L.k64.t, st));
        SGOC_LAUNCH(launch_sub(L.k64.b, L.k64.t, L.k64.r, N, st));
        SGOC_TRY(norm2(L.k64.r, N, L.k64.partial, L.k64.scal, &rn, st));
      }
      rel = rn / bnorm;
      *rel_out = rel;
      if (rel <= pb->opt.tol || hs.flag == 2) return SGOC_OK;
      target *= pb->opt.tol / rel;
      const int zero = 0;
      SGOC_CUDA_TRY(cudaMemcpyAsync(&L.k64.state->target, &target, sizeof(double), cudaMemcpyHostToDevice, st));
      SGOC_CUDA_TRY(cudaMemcpyAsync(&L.k64.state->flag, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
      SGOC_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
  set_error("MINRES iteration limit reached");
  return SGOC_ERR_NO_CONVERGENCE;
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

static sgoc_status solve_impl(sgoc_problem* pb, void* d_ws, size_t ws_bytes, const double* d_x0, double* d_x,
                              cudaStream_t st, sgoc_result* res) {
  Layout L;
  const int prec = pb->opt.precision;
  carve_layout(pb, prec, d_ws, ws_bytes, L);
  const int64_t N = pb->N;
  SGOC_TRY(rhs_apply(pb, L.k64.b, st));
  double bnorm = 0;
  SGOC_TRY(norm2(L.k64.b, N, L.k64.partial, L.k64.scal, &bnorm, st));
  if (res) { res->iterations = 0; res->outer_iterations = 0; res->rel_true_residual = 0; res->rel_estimate = 0; }
  if (d_x0) SGOC_CUDA_TRY(cudaMemcpyAsync(d_x, d_x0, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else SGOC_LAUNCH(launch_fill<double>(d_x, N, 0.0, st));
  if (bnorm == 0.0) { SGOC_LAUNCH(launch_fill<double>(d_x, N, 0.0, st)); SGOC_CUDA_TRY(cudaStreamSynchronize(st)); return SGOC_OK; }
  if (!std::isfinite(bnorm)) { set_error("non-finite right-hand side"); return SGOC_ERR_NAN; }

  if (prec == SGOC_FP64) {
    // r0 = b - K x0; the stopping rule is relative to b, so with an initial guess
    // the estimate target is rescaled by ||b|| / ||r0|| (2-norms) and the true
    // residual decides at exit
    const double* rhs = L.k64.b;
    double target = pb->opt.tol;
    if (d_x0) {
      SGOC_TRY(kkt_apply<double>(pb, d_x, L.k64.t, st));
      SGOC_LAUNCH(launch_sub(L.k64.b, L.k64.t, L.k64.r, N, st));
      double rn0 = 0;
      SGOC_TRY(norm2(L.k64.r, N, L.k64.partial, L.k64.scal, &rn0, st));
      if (res) { res->iterations = 0; res->outer_iterations = 0; res->rel_true_residual = rn0 / bnorm; }
      if (rn0 / bnorm <= pb->opt.tol) return SGOC_OK;
      target = std::min(0.5, pb->opt.tol * bnorm / rn0);
      rhs = L.k64.r;
    }
    int it = 0; double est = 1, rel = 1;
    sgoc_status s = minres<double>(pb, L, L.m64, rhs, d_x, target, pb->opt.max_iter, true, bnorm, st, &it,
                                   &est, &rel);
    if (res) { res->iterations = it; res->outer_iterations = 1; res->rel_estimate = est; res->rel_true_residual = rel; }
    return s;
  }
  // mixed: float32 inner MINRES inside float64 iterative refinement
  int total = 0;
  double rel = 1, est = 1;
  for (int k = 0; k < pb->opt.max_outer; ++k) {
    SGOC_TRY(kkt_apply<double>(pb, d_x, L.k64.t, st));
    SGOC_LAUNCH(launch_sub(L.k64.b, L.k64.t, L.k64.r, N, st));
    double rn = 0;
    SGOC_TRY(norm2(L.k64.r, N, L.k64.partial, L.k64.scal, &rn, st));
    rel = rn / bnorm;
    if (res) { res->outer_iterations = k; res->rel_true_residual = rel; res->iterations = total; }
    if (!std::isfinite(rel)) { set_error("non-finite residual in refinement"); return SGOC_ERR_NAN; }
    if (rel <= pb->opt.tol) return SGOC_OK;
    // unit-norm residual in float32, inner solve K c = r / ||r||, then x += ||r|| c
    SGOC_LAUNCH(launch_scale_to32(L.k64.r, L.rhs32, N, 1.0 / rn, st));
    SGOC_LAUNCH(launch_fill<float>(L.c32, N, 0.0f, st));
    int it = 0;
    double unused = 0;
    sgoc_status s = minres<float>(pb, L, L.m32, L.rhs32, L.c32, pb->opt.inner_tol, pb->opt.max_iter, false, 1.0,
                                  st, &it, &est, &unused);
    total += it;
    if (s != SGOC_OK && s != SGOC_ERR_NO_CONVERGENCE) return s;
    SGOC_LAUNCH(launch_add_scaled(L.c32, d_x, N, rn, st));
    if (res) { res->iterations = total; res->rel_estimate = est; res->outer_iterations = k + 1; }
  }
  set_error("iterative refinement step limit reached");
  return SGOC_ERR_NO_CONVERGENCE;
}

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

sgoc_status sgoc_rhs(sgoc_problem* pb, double* d_b, void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_b) { set_error("null output"); return SGOC_ERR_INVALID_ARG; }
  return rhs_apply(pb, d_b, static_cast<cudaStream_t>(stream));
}

sgoc_status sgoc_solve(sgoc_problem* pb, void* d_ws, size_t ws_bytes, const double* d_x0, double* d_x,
                       void* stream, sgoc_result* res) {
  auto t0 = std::chrono::steady_clock::now();
  SGOC_TRY(check_ready(pb));
  if (!d_x) { set_error("null solution buffer"); return SGOC_ERR_INVALID_ARG; }
  SGOC_TRY(check_ws(d_ws, ws_bytes, workspace_bytes(pb, pb->opt.precision)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  sgoc_status s = solve_impl(pb, d_ws, ws_bytes, d_x0, d_x, st, res);
  cudaError_t e = cudaStreamSynchronize(st);
  if (s == SGOC_OK && e != cudaSuccess) s = cuda_status(e, "cudaStreamSynchronize");
  if (res) {
    res->status = s;
    res->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}

sgoc_status sgoc_apply_operator(sgoc_problem* pb, int32_t precision, const void* d_X, void* d_Y, int32_t nslabs,
                                void* stream) {
  SGOC_TRY(check_ready(pb));
  if (!d_X || !d_Y || nslabs < 1) { set_error("bad arguments"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
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

}  // extern "C"
