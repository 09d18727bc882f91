// Host set-up of an SG optimal-control problem: validation, chaos basis,
// triple-product tables, multigrid hierarchy of the mean operator, and the
// upload of the coefficient data into the caller's persistent device buffer.
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "kernels.h"
#include "sgoc_internal.h"

namespace sgoc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// Graded multi-index set, lexicographically descending inside each degree
// (degree 1 is e_1, ..., e_M): the level structure swept by Alg. 1.
static void gen_degree(int M, int pos, int remaining, std::vector<int32_t>& cur,
                       std::vector<int32_t>& out) {
  if (pos == M - 1) {
    cur[pos] = remaining;
    out.insert(out.end(), cur.begin(), cur.end());
    return;
  }
  for (int v = remaining; v >= 0; --v) {
    cur[pos] = v;
    gen_degree(M, pos + 1, remaining - v, cur, out);
  }
}

static double binom(int a, int b) {
  if (b < 0 || b > a) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
  return r;
}

// E[psi_a psi_b psi_c] for normalised Hermite polynomials psi_n = He_n / sqrt(n!), xi ~ N(0,1):
// sqrt(a! b! c!) / ((s-a)! (s-b)! (s-c)!) for even a+b+c = 2s with s >= max(a, b, c), else 0.
static double hermite_triple(int a, int b, int c) {
  if ((a + b + c) % 2) return 0.0;
  const int s = (a + b + c) / 2;
  if (s < std::max(a, std::max(b, c))) return 0.0;
  auto fact = [](int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; };
  return std::sqrt(fact(a) * fact(b) * fact(c)) / (fact(s - a) * fact(s - b) * fact(s - c));
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace sgoc

using namespace sgoc;

extern "C" {

const char* sgoc_last_error(void) { return g_last_error.c_str(); }

const char* sgoc_status_string(sgoc_status s) {
  switch (s) {
    case SGOC_OK: return "ok";
    case SGOC_ERR_INVALID_ARG: return "invalid argument";
    case SGOC_ERR_UNSUPPORTED: return "unsupported problem";
    case SGOC_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case SGOC_ERR_CUDA: return "CUDA error";
    case SGOC_ERR_NO_CONVERGENCE: return "no convergence";
    case SGOC_ERR_BREAKDOWN: return "Lanczos breakdown";
    case SGOC_ERR_NOT_SPD: return "preconditioner not positive definite";
    case SGOC_ERR_NAN: return "NaN or Inf";
    case SGOC_ERR_NOT_UPLOADED: return "problem data not uploaded";
  }
  return "unknown status";
}

void sgoc_default_options(sgoc_options* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->max_iter = 1000;
  o->r = 0;
  o->cheb_steps = 5;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->omega = 0.8;
  o->precision = SGOC_FP64;
  o->inner_tol = 1e-3;
  o->max_outer = 20;
  o->schur = 0;
  o->krylov = 0;
  o->restart = 64;
  o->mass_solve = 0;
  o->precond = 0;
  o->mean_solve = 0;
}

namespace sgoc {
// Slot table of one SG launch shape (see UTab): which (alpha, k) products
// sum_e kappa_k(e) T_e(alpha) the outputs of the shape use, and where each
// output finds them.  Entries keep the order of the neighbour table.
// Neighbour table of the output columns: the full one or its downward part (entries
// whose input column lies one level below the output's).
struct NbrView {
  const std::vector<int>& ptr;
  const std::vector<int>& alpha;
  const std::vector<int>& k;
  const std::vector<double>& c;
};

// own: the outputs also use their own columns (kappa_0 term); then (beta, 0) has a slot.
static UTab build_utab(const NbrView& t, int in0, int in1, int out0, int out1, int kmax, bool own) {
  UTab u;
  u.in0 = in0; u.in1 = in1; u.out0 = out0; u.out1 = out1; u.kmax = kmax;
  const int nin = in1 - in0, nout = out1 - out0;
  std::vector<unsigned> mask(nin, 0u);
  auto end_of = [&](int b) {
    int e = t.ptr[b];
    while (e < t.ptr[b + 1] && t.k[e] < kmax) ++e;
    return e;
  };
  for (int b = out0; b < out1; ++b) {
    if (own) mask[b - in0] |= 1u;
    for (int e = t.ptr[b]; e < end_of(b); ++e) mask[t.alpha[e] - in0] |= 1u << t.k[e];
  }
  u.mb.resize(2 * size_t(nin));
  int base = 0;
  for (int c = 0; c < nin; ++c) {
    u.mb[2 * c] = int(mask[c]);
    u.mb[2 * c + 1] = base;
    base += __builtin_popcount(mask[c]);
  }
  u.nslots = base;
  auto slot = [&](int a, int k) {
    const unsigned m = mask[a - in0];
    return u.mb[2 * (a - in0) + 1] + __builtin_popcount(m & ((1u << k) - 1u));
  };
  u.diag.resize(nout);
  u.eptr.assign(nout + 1, 0);
  for (int b = out0; b < out1; ++b) {
    u.diag[b - out0] = own ? slot(b, 0) : -1;
    for (int e = t.ptr[b]; e < end_of(b); ++e) {
      u.eslot.push_back(slot(t.alpha[e], t.k[e]));
      u.ec.push_back(t.c[e]);
    }
    u.eptr[b - out0 + 1] = int(u.eslot.size());
  }
  u.nent = int(u.eslot.size());
  return u;
}

static size_t utab_bytes(const UTab& u) {
  const size_t nin = u.in1 - u.in0, nout = u.out1 - u.out0;
  return align256(nin * 8) + align256(nout * 4) + align256((nout + 1) * 4) + align256(size_t(u.nent) * 8) +
         align256(size_t(u.nent) * 4) + align256(size_t(u.nent) * 8);
}
}  // namespace sgoc

sgoc_status sgoc_problem_create(const sgoc_problem_desc* d, const sgoc_options* opt,
                                sgoc_problem** out) {
  if (!d || !out) { set_error("null desc/out"); return SGOC_ERR_INVALID_ARG; }
  *out = nullptr;
  const int nx = d->nx;
  if (nx < 2 || nx > 4096 || (nx & (nx - 1)) != 0) {
    set_error("nx must be a power of two in [2, 4096]");
    return (nx >= 2 && nx <= 4096) ? SGOC_ERR_UNSUPPORTED : SGOC_ERR_INVALID_ARG;
  }
  if (d->M < 0 || d->M > 16 || d->p < 0 || d->p > 10) { set_error("M in [0,16], p in [0,10]"); return SGOC_ERR_INVALID_ARG; }
  if (!(d->beta > 0.0) || !(d->gamma >= 0.0) || !std::isfinite(d->beta) || !std::isfinite(d->gamma)) {
    set_error("beta > 0 and gamma >= 0 required"); return SGOC_ERR_INVALID_ARG;
  }
  if (d->nt < 0 || d->nt > 100000 || (d->nt > 0 && !(d->T > 0.0))) { set_error("nt >= 0, T > 0"); return SGOC_ERR_INVALID_ARG; }
  if (!d->kappa || !d->yhat) { set_error("kappa and yhat are required"); return SGOC_ERR_INVALID_ARG; }
  const double Pd = binom(d->M + d->p, d->p);
  if (d->chaos != 0 && d->chaos != 1) { set_error("chaos must be 0 (Legendre) or 1 (Hermite)"); return SGOC_ERR_INVALID_ARG; }
  const double length = d->length == 0.0 ? 1.0 : d->length;
  if (!(length > 0) || !std::isfinite(length)) { set_error("domain length must be positive"); return SGOC_ERR_INVALID_ARG; }
  const double nterms_d = d->chaos == 1 ? binom(d->M + 2 * d->p, 2 * d->p) : double(d->M + 1);
  if (nterms_d > 20000) { set_error("too many coefficient terms"); return SGOC_ERR_INVALID_ARG; }
  const int nterms = int(nterms_d + 0.5);
  if (Pd > 20000) { set_error("chaos basis too large (P > 20000)"); return SGOC_ERR_UNSUPPORTED; }
  sgoc_options o;
  sgoc_default_options(&o);
  if (opt) o = *opt;
  if (o.r == 0) o.r = d->M + 1;
  if (o.r < 1 || o.r > nterms) { set_error("truncation r must be in [1, n_terms]"); return SGOC_ERR_INVALID_ARG; }
  if (!(o.tol > 0) || o.max_iter < 1 || o.cheb_steps < 1 || o.cheb_steps > 64 || o.nu_pre < 0 || o.nu_post < 0 ||
      o.nu_pre > 16 || o.nu_post > 16 || o.nu_pre != o.nu_post || !(o.omega > 0 && o.omega < 2) ||
      (o.precision != SGOC_FP64 && o.precision != SGOC_MIXED_FP32) || !(o.inner_tol > 0 && o.inner_tol < 1) ||
      o.max_outer < 1 || (o.schur != 0 && o.schur != 1) || (o.krylov != 0 && o.krylov != 1) ||
      o.restart < 1 || o.restart > kFgmresMax || (o.mass_solve != 0 && o.mass_solve != 1) ||
      (o.precond != 0 && o.precond != 1) || (o.precond == 1 && o.krylov != 1) ||
      (o.mean_solve != 0 && o.mean_solve != 1)) {
    set_error("invalid options (nu_pre must equal nu_post for a symmetric V-cycle)");
    return SGOC_ERR_INVALID_ARG;
  }

  if (o.mean_solve != 0 && (o.precision != SGOC_MIXED_FP32 || !spectral_mean_supported(nx - 1))) {
    set_error("exact mean solves (mean_solve = 1) need mixed precision and nx = 64 or 128");
    return SGOC_ERR_UNSUPPORTED;
  }

  auto* pb = new sgoc_problem();
  pb->nx = nx; pb->M = d->M; pb->p = d->p; pb->nt = d->nt;
  pb->chaos = d->chaos; pb->nterms = nterms; pb->length = length;
  pb->beta = d->beta; pb->gamma = d->gamma; pb->T = d->T;
  pb->tau = d->nt > 0 ? d->T / d->nt : 1.0;
  pb->n1 = nx - 1;
  pb->n = int64_t(pb->n1) * pb->n1;
  pb->P = int(Pd + 0.5);
  pb->slabs = d->nt > 0 ? d->nt : 1;
  pb->F = int64_t(pb->slabs) * pb->P * pb->n;
  pb->N = 3 * pb->F;
  pb->opt = o;
  pb->r = o.r;
  pb->s = std::sqrt((1.0 + d->gamma) / d->beta);

  const int64_t nel = int64_t(nx) * nx;
  pb->kappa.assign(d->kappa, d->kappa + int64_t(nterms) * nel);
  for (double v : pb->kappa)
    if (!std::isfinite(v)) { delete pb; set_error("non-finite kappa"); return SGOC_ERR_NAN; }
  pb->kappa0 = pb->kappa[0];
  for (int64_t e = 0; e < nel; ++e)
    if (pb->kappa[e] != pb->kappa0) {
      delete pb;
      set_error("kappa_0 (the mean field) must be spatially constant");
      return SGOC_ERR_UNSUPPORTED;
    }
  if (!(pb->kappa0 > 0)) { delete pb; set_error("kappa_0 must be positive"); return SGOC_ERR_INVALID_ARG; }
  pb->yhat.assign(d->yhat, d->yhat + int64_t(pb->slabs) * pb->n);
  for (double v : pb->yhat)
    if (!std::isfinite(v)) { delete pb; set_error("non-finite yhat"); return SGOC_ERR_NAN; }
  if (d->nt > 0 && d->y0) {
    pb->y0.assign(d->y0, d->y0 + pb->n);
    for (double v : pb->y0)
      if (!std::isfinite(v)) { delete pb; set_error("non-finite y0"); return SGOC_ERR_NAN; }
  }

  // chaos multi-indices, graded
  const int M = d->M, p = d->p;
  if (M > 0) {
    std::vector<int32_t> cur(M, 0);
    for (int deg = 0; deg <= p; ++deg) gen_degree(M, 0, deg, cur, pb->idx);
  }
  pb->off.resize(p + 2);
  pb->off[0] = 0;
  for (int deg = 0; deg <= p; ++deg) pb->off[deg + 1] = int(binom(M + deg, deg) + 0.5);
  if (M > 0 && int64_t(pb->idx.size()) != int64_t(pb->P) * M) {
    delete pb; set_error("internal: multi-index count"); return SGOC_ERR_INVALID_ARG;
  }
  // the register SG kernel's compiled multi-index order must be this one
  {
    std::vector<int> tab;
    pb->sgr_ok = d->chaos == 0 && M > 0 && sgr_indices(M, p, tab) &&
                 tab == std::vector<int>(pb->idx.begin(), pb->idx.end());
  }
  // neighbour table of G_k: beta couples to beta + e_k and beta - e_k
  std::map<std::vector<int32_t>, int> pos;
  for (int a = 0; a < pb->P && M > 0; ++a)
    pos[std::vector<int32_t>(pb->idx.begin() + int64_t(a) * M, pb->idx.begin() + int64_t(a + 1) * M)] = a;
  pb->nbr_ptr.assign(pb->P + 1, 0);
  if (d->chaos == 1 && M > 0) {
    // Hermite: beta couples to alpha through term l >= 1 with c = E[psi_l Psi_alpha Psi_beta]
    // = prod_j e(alpha_j, beta_j, l_j) (the closed form of hermite_triple), entries by l, then alpha
    std::vector<int32_t> cur(M, 0);
    for (int deg = 0; deg <= 2 * p; ++deg) gen_degree(M, 0, deg, cur, pb->tidx);
    if (int64_t(pb->tidx.size()) != int64_t(nterms) * M) { delete pb; set_error("internal: term count"); return SGOC_ERR_INVALID_ARG; }
    for (int b = 0; b < pb->P; ++b) {
      for (int l = 1; l < nterms; ++l) {
        for (int a = 0; a < pb->P; ++a) {
          double c = 1.0;
          for (int j = 0; j < M && c != 0.0; ++j)
            c *= hermite_triple(pb->idx[int64_t(a) * M + j], pb->idx[int64_t(b) * M + j], pb->tidx[int64_t(l) * M + j]);
          if (c != 0.0) { pb->nbr_alpha.push_back(a); pb->nbr_k.push_back(l); pb->nbr_c.push_back(c); }
        }
      }
      pb->nbr_ptr[b + 1] = int(pb->nbr_alpha.size());
    }
  }
  for (int b = 0; b < pb->P && d->chaos == 0; ++b) {
    for (int k = 0; k < M; ++k) {
      std::vector<int32_t> v(pb->idx.begin() + int64_t(b) * M, pb->idx.begin() + int64_t(b + 1) * M);
      const int bk = v[k];
      if (bk >= 1) {
        v[k] = bk - 1;
        auto it = pos.find(v);
        if (it != pos.end()) {
          pb->nbr_alpha.push_back(it->second); pb->nbr_k.push_back(k + 1);
          pb->nbr_c.push_back(legendre_coupling(bk - 1));
        }
      }
      v[k] = bk + 1;
      auto it = pos.find(v);
      if (it != pos.end()) {
        pb->nbr_alpha.push_back(it->second); pb->nbr_k.push_back(k + 1);
        pb->nbr_c.push_back(legendre_coupling(bk));
      }
    }
    pb->nbr_ptr[b + 1] = int(pb->nbr_alpha.size());
  }
  // end of each column's entries with k < r (the table is sorted by k inside a column)
  pb->nbr_end_r.resize(pb->P);
  for (int b = 0; b < pb->P; ++b) {
    int e = pb->nbr_ptr[b];
    while (e < pb->nbr_ptr[b + 1] && pb->nbr_k[e] < pb->r) ++e;
    pb->nbr_end_r[b] = e;
  }
  // downward part: entries alpha = beta - e_k one level below beta (the only nonzero couplings of a
  // level's first hGS visit, when the levels at and above it are still zero)
  std::vector<int> level_of(pb->P);
  for (int d = 0; d <= p; ++d)
    for (int b = pb->off[d]; b < pb->off[d + 1]; ++b) level_of[b] = d;
  pb->dn_ptr.assign(pb->P + 1, 0);
  pb->dn_end_r.resize(pb->P);
  for (int b = 0; b < pb->P; ++b) {
    for (int e = pb->nbr_ptr[b]; e < pb->nbr_ptr[b + 1]; ++e)
      if (level_of[pb->nbr_alpha[e]] < level_of[b]) {
        pb->dn_alpha.push_back(pb->nbr_alpha[e]);
        pb->dn_k.push_back(pb->nbr_k[e]);
        pb->dn_c.push_back(pb->nbr_c[e]);
      }
    pb->dn_ptr[b + 1] = int(pb->dn_alpha.size());
    int e = pb->dn_ptr[b];
    while (e < pb->dn_ptr[b + 1] && pb->dn_k[e] < pb->r) ++e;
    pb->dn_end_r[b] = e;
  }
  // input levels an hGS visit reads: the largest level distance of a kept coupling (1 for
  // Legendre: G_k couples neighbouring levels only)
  pb->lev_dist = 1;
  for (int b = 0; b < pb->P; ++b)
    for (int e = pb->nbr_ptr[b]; e < pb->nbr_end_r[b]; ++e)
      pb->lev_dist = std::max(pb->lev_dist, std::abs(level_of[pb->nbr_alpha[e]] - level_of[b]));

  // multigrid hierarchy of the mean operator:
  // steady  A~_1 = kappa0 K + s M            (Eq. (mathcalZ))
  // time    A^_1 = (1 + tau s) M + tau kappa0 K  (Eq. (A_hat))
  // Q1 on a uniform grid: K stencil (1/3)[-1 -1 -1; -1 8 -1; -1 -1 -1], M = h^2/36 [1 4 1; 4 16 4; 1 4 1];
  // Galerkin coarse operators of nested Q1 spaces are the coarse-grid Q1 matrices.
  const double ck = d->nt > 0 ? pb->tau * pb->kappa0 : pb->kappa0;
  const double cm = d->nt > 0 ? 1.0 + pb->tau * pb->s : pb->s;
  for (int g = nx; g >= 2; g /= 2) {
    Level L;
    L.nx = g; L.n1 = g - 1; L.n = int64_t(L.n1) * L.n1;
    const double h = length / g, m = h * h / 36.0;
    L.diag = ck * (8.0 / 3.0) + cm * 16.0 * m;
    L.edge = -ck / 3.0 + cm * 4.0 * m;
    L.corner = -ck / 3.0 + cm * m;
    pb->levels.push_back(L);
  }
  pb->mass_h2_36 = length * length / (36.0 * nx * double(nx));
  pb->dweights.assign(pb->slabs, 1.0);
  if (d->nt > 1) { pb->dweights[0] = 0.5; pb->dweights[d->nt - 1] = 0.5; }

  // slot tables of the SG launch shapes: the full operator and the hGS visit of each level
  const NbrView full{pb->nbr_ptr, pb->nbr_alpha, pb->nbr_k, pb->nbr_c};
  const NbrView down{pb->dn_ptr, pb->dn_alpha, pb->dn_k, pb->dn_c};
  // (the two-phase kernel keeps one mask bit per coefficient term: at most 17 terms)
  const int D = pb->lev_dist;
  auto lo = [&](int d) { return pb->off[std::max(0, d - D)]; };
  auto hi = [&](int d) { return pb->off[std::min(p + 1, d + D + 1)]; };
  const bool slots = nterms <= 17;
  pb->utabs.push_back(slots ? build_utab(full, 0, pb->P, 0, pb->P, nterms, true) : UTab());
  for (int d = 0; d <= p; ++d)
    pb->utabs.push_back(slots ? build_utab(full, lo(d), hi(d), pb->off[d], pb->off[d + 1], pb->r, true) : UTab());
  for (int d = 0; d <= p; ++d)
    pb->utabs.push_back(slots ? build_utab(down, lo(d), pb->off[d], pb->off[d], pb->off[d + 1], pb->r, false) : UTab());

  // persistent layout
  const size_t nk = size_t(nterms) * nel;
  const size_t nnz = pb->nbr_alpha.size();
  size_t off = 0;
  off = align256(off + nk * 8); off = align256(off + nk * 4);
  off = align256(off + (pb->P + 1) * 4); off = align256(off + nnz * 4); off = align256(off + nnz * 4);
  off = align256(off + pb->P * 4);
  off = align256(off + nnz * 8); off = align256(off + nnz * 4);
  off = align256(off + size_t(pb->slabs) * pb->n * 8); off = align256(off + size_t(pb->n) * 8);
  const size_t nnz_dn = pb->dn_alpha.size();
  off = align256(off + (pb->P + 1) * 4); off = align256(off + pb->P * 4); off = align256(off + nnz_dn * 4);
  off = align256(off + nnz_dn * 4); off = align256(off + nnz_dn * 8); off = align256(off + nnz_dn * 4);
  for (const UTab& u : pb->utabs) off += utab_bytes(u);
  off += 2 * align256(size_t(pb->n1) * 8) + 2 * align256(size_t(pb->n1) * 4);   // mass factor tables
  // the fast-diagonalisation image: exact mean solves, and exact mass blocks in float32
  pb->spec = o.precision == SGOC_MIXED_FP32 && spectral_mean_supported(pb->n1) &&
             (o.mean_solve != 0 || o.mass_solve == 1);
  if (pb->spec) off += align256(spectral_image_bytes(pb->n1));
  pb->persistent_bytes = off;
  *out = pb;
  return SGOC_OK;
}

void sgoc_problem_destroy(sgoc_problem* pb) {
  if (!pb) return;
  release_runtime(pb);
  delete pb;
}

sgoc_status sgoc_problem_sizes(const sgoc_problem* pb, int64_t* n, int64_t* P, int64_t* slabs,
                               int64_t* kkt) {
  if (!pb) { set_error("null problem"); return SGOC_ERR_INVALID_ARG; }
  if (n) *n = pb->n;
  if (P) *P = pb->P;
  if (slabs) *slabs = pb->slabs;
  if (kkt) *kkt = pb->N;
  return SGOC_OK;
}

sgoc_status sgoc_problem_device_bytes(const sgoc_problem* pb, size_t* persistent, size_t* workspace) {
  if (!pb) { set_error("null problem"); return SGOC_ERR_INVALID_ARG; }
  if (persistent) *persistent = pb->persistent_bytes;
  if (workspace) *workspace = workspace_bytes(pb, pb->opt.precision);
  return SGOC_OK;
}

sgoc_status sgoc_problem_upload(sgoc_problem* pb, void* d_persistent, size_t bytes, void* stream) {
  if (!pb || !d_persistent) { set_error("null problem/buffer"); return SGOC_ERR_INVALID_ARG; }
  if (bytes < pb->persistent_bytes) { set_error("persistent buffer too small"); return SGOC_ERR_WORKSPACE_TOO_SMALL; }
  if (reinterpret_cast<uintptr_t>(d_persistent) % 256) { set_error("persistent buffer must be 256-byte aligned"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  invalidate_graphs(pb);
  const size_t nel = size_t(pb->nx) * pb->nx, nk = size_t(pb->nterms) * nel;
  const size_t nnz = pb->nbr_alpha.size();
  char* base = static_cast<char*>(d_persistent);
  size_t off = 0;
  auto carve = [&](size_t b) { char* p = base + off; off = align256(off + b); return p; };
  pb->dev.kap64 = reinterpret_cast<double*>(carve(nk * 8));
  pb->dev.kap32 = reinterpret_cast<float*>(carve(nk * 4));
  pb->dev.nbr_ptr = reinterpret_cast<int*>(carve((pb->P + 1) * 4));
  pb->dev.nbr_end_all = pb->dev.nbr_ptr + 1;                     // all entries: the next column's start
  pb->dev.nbr_end_r = reinterpret_cast<int*>(carve(pb->P * 4));
  pb->dev.nbr_alpha = reinterpret_cast<int*>(carve(nnz * 4));
  pb->dev.nbr_k = reinterpret_cast<int*>(carve(nnz * 4));
  pb->dev.nbr_c64 = reinterpret_cast<double*>(carve(nnz * 8));
  pb->dev.nbr_c32 = reinterpret_cast<float*>(carve(nnz * 4));
  pb->dev.yhat = reinterpret_cast<double*>(carve(size_t(pb->slabs) * pb->n * 8));
  pb->dev.y0 = reinterpret_cast<double*>(carve(size_t(pb->n) * 8));
  const size_t nnz_dn = pb->dn_alpha.size();
  pb->dev.dn_ptr = reinterpret_cast<int*>(carve((pb->P + 1) * 4));
  pb->dev.dn_end_r = reinterpret_cast<int*>(carve(pb->P * 4));
  pb->dev.dn_alpha = reinterpret_cast<int*>(carve(nnz_dn * 4));
  pb->dev.dn_k = reinterpret_cast<int*>(carve(nnz_dn * 4));
  pb->dev.dn_c64 = reinterpret_cast<double*>(carve(nnz_dn * 8));
  pb->dev.dn_c32 = reinterpret_cast<float*>(carve(nnz_dn * 4));
  std::vector<float> dn32(pb->dn_c.begin(), pb->dn_c.end());
  std::vector<std::vector<int2>> e32s;
  for (UTab& u : pb->utabs) {
    const size_t nin = u.in1 - u.in0, nout = u.out1 - u.out0;
    u.d_mb = reinterpret_cast<int*>(carve(nin * 8));
    u.d_diag = reinterpret_cast<int*>(carve(nout * 4));
    u.d_eptr = reinterpret_cast<int*>(carve((nout + 1) * 4));
    u.d_e32 = reinterpret_cast<int2*>(carve(size_t(u.nent) * 8));
    u.d_eslot = reinterpret_cast<int*>(carve(size_t(u.nent) * 4));
    u.d_ec64 = reinterpret_cast<double*>(carve(size_t(u.nent) * 8));
    std::vector<int2> e32(u.nent);
    for (int i = 0; i < u.nent; ++i) {
      const float c = float(u.ec[i]);
      int bits;
      std::memcpy(&bits, &c, 4);
      e32[i] = make_int2(u.eslot[i] * 32, bits);            // offset of the slot's row of 32 nodes
    }
    e32s.push_back(std::move(e32));
  }

  pb->dev.mass_l64 = reinterpret_cast<double*>(carve(size_t(pb->n1) * 8));
  pb->dev.mass_id64 = reinterpret_cast<double*>(carve(size_t(pb->n1) * 8));
  pb->dev.mass_l32 = reinterpret_cast<float*>(carve(size_t(pb->n1) * 4));
  pb->dev.mass_id32 = reinterpret_cast<float*>(carve(size_t(pb->n1) * 4));
  // M1 = a tridiag(1, 4, 1), a = h/6: D_0 = 4a, l_i = a / D_{i-1}, D_i = 4a - a l_i
  std::vector<double> l(pb->n1, 0.0), id(pb->n1);
  std::vector<float> l32, id32;
  {
    const double a = pb->length / (6.0 * pb->nx);
    double D = 4.0 * a;
    id[0] = 1.0 / D;
    for (int i = 1; i < pb->n1; ++i) {
      l[i] = a / D;
      D = 4.0 * a - a * l[i];
      id[i] = 1.0 / D;
    }
    l32.assign(l.begin(), l.end());
    id32.assign(id.begin(), id.end());
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.mass_l64, l.data(), l.size() * 8, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.mass_id64, id.data(), id.size() * 8, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.mass_l32, l32.data(), l32.size() * 4, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.mass_id32, id32.data(), id32.size() * 4, cudaMemcpyHostToDevice, st));
  }
  // constant image of the exact mean solves: split sine-transform operands and mode table
  std::vector<uint8_t> spec;
  pb->dev.spec_img = nullptr;
  if (pb->spec) {
    spec = spectral_image(pb->n1);
    pb->dev.spec_img = carve(spec.size());
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.spec_img, spec.data(), spec.size(), cudaMemcpyHostToDevice, st));
  }
  std::vector<double> k64(nk);
  std::vector<float> k32(nk);
  for (size_t i = 0; i < nk; ++i) { k64[i] = pb->kappa[i] / 6.0; k32[i] = float(k64[i]); }
  std::vector<float> c32(pb->nbr_c.begin(), pb->nbr_c.end());
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.kap64, k64.data(), nk * 8, cudaMemcpyHostToDevice, st));
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.kap32, k32.data(), nk * 4, cudaMemcpyHostToDevice, st));
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.nbr_ptr, pb->nbr_ptr.data(), (pb->P + 1) * 4, cudaMemcpyHostToDevice, st));
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.nbr_end_r, pb->nbr_end_r.data(), pb->P * 4, cudaMemcpyHostToDevice, st));
  if (nnz) {
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.nbr_alpha, pb->nbr_alpha.data(), nnz * 4, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.nbr_k, pb->nbr_k.data(), nnz * 4, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.nbr_c64, pb->nbr_c.data(), nnz * 8, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.nbr_c32, c32.data(), nnz * 4, cudaMemcpyHostToDevice, st));
  }
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.yhat, pb->yhat.data(), size_t(pb->slabs) * pb->n * 8,
                                cudaMemcpyHostToDevice, st));
  if (!pb->y0.empty())
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.y0, pb->y0.data(), size_t(pb->n) * 8, cudaMemcpyHostToDevice, st));
  else
    SGOC_CUDA_TRY(cudaMemsetAsync(pb->dev.y0, 0, size_t(pb->n) * 8, st));
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.dn_ptr, pb->dn_ptr.data(), (pb->P + 1) * 4, cudaMemcpyHostToDevice, st));
  SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.dn_end_r, pb->dn_end_r.data(), pb->P * 4, cudaMemcpyHostToDevice, st));
  if (nnz_dn) {
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.dn_alpha, pb->dn_alpha.data(), nnz_dn * 4, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.dn_k, pb->dn_k.data(), nnz_dn * 4, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.dn_c64, pb->dn_c.data(), nnz_dn * 8, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(pb->dev.dn_c32, dn32.data(), nnz_dn * 4, cudaMemcpyHostToDevice, st));
  }
  for (size_t i = 0; i < pb->utabs.size(); ++i) {
    const UTab& u = pb->utabs[i];
    if (u.eptr.empty()) continue;                 // no slot table (more than 17 coefficient terms)
    const size_t nin = u.in1 - u.in0, nout = u.out1 - u.out0;
    SGOC_CUDA_TRY(cudaMemcpyAsync(u.d_mb, u.mb.data(), nin * 8, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(u.d_diag, u.diag.data(), nout * 4, cudaMemcpyHostToDevice, st));
    SGOC_CUDA_TRY(cudaMemcpyAsync(u.d_eptr, u.eptr.data(), (nout + 1) * 4, cudaMemcpyHostToDevice, st));
    if (u.nent) {
      SGOC_CUDA_TRY(cudaMemcpyAsync(u.d_e32, e32s[i].data(), size_t(u.nent) * 8, cudaMemcpyHostToDevice, st));
      SGOC_CUDA_TRY(cudaMemcpyAsync(u.d_eslot, u.eslot.data(), size_t(u.nent) * 4, cudaMemcpyHostToDevice, st));
      SGOC_CUDA_TRY(cudaMemcpyAsync(u.d_ec64, u.ec.data(), size_t(u.nent) * 8, cudaMemcpyHostToDevice, st));
    }
  }
  // the host vectors above go out of scope: finish the copies first
  SGOC_CUDA_TRY(cudaStreamSynchronize(st));
  pdl_fence(st);
  pb->uploaded = true;
  return SGOC_OK;
}

sgoc_status sgoc_pc_indices(const sgoc_problem* pb, int32_t* host_out) {
  if (!pb || (!host_out && pb->M > 0)) { set_error("null argument"); return SGOC_ERR_INVALID_ARG; }
  if (pb->M > 0) std::memcpy(host_out, pb->idx.data(), pb->idx.size() * sizeof(int32_t));
  return SGOC_OK;
}

sgoc_status sgoc_triple_products(const sgoc_problem* pb, int32_t* k, int32_t* a, int32_t* b,
                                 double* c, int64_t* nnz) {
  if (!pb || !nnz) { set_error("null argument"); return SGOC_ERR_INVALID_ARG; }
  const int64_t cnt = int64_t(pb->nbr_alpha.size());
  if (!k && !a && !b && !c) { *nnz = cnt; return SGOC_OK; }
  if (!k || !a || !b || !c) { set_error("all output arrays are required"); return SGOC_ERR_INVALID_ARG; }
  if (*nnz < cnt) { *nnz = cnt; set_error("capacity too small"); return SGOC_ERR_INVALID_ARG; }
  int64_t q = 0;
  for (int beta = 0; beta < pb->P; ++beta)
    for (int e = pb->nbr_ptr[beta]; e < pb->nbr_ptr[beta + 1]; ++e, ++q) {
      k[q] = pb->nbr_k[e]; a[q] = pb->nbr_alpha[e]; b[q] = beta; c[q] = pb->nbr_c[e];
    }
  *nnz = cnt;
  return SGOC_OK;
}

}  // extern "C"
