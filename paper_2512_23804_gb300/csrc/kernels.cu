// Device kernels of the SG optimal-control solver (sm_103a).
//
// Grid conventions: interior nodes (ix, iy), 0 <= ix, iy < n1 = nx - 1, node index
// iy*n1 + ix; element (ex, ey), 0 <= ex, ey < nx.  Interior node (ix, iy) is the
// north-east corner of element (ix, iy), the north-west corner of (ix+1, iy), the
// south-west corner of (ix+1, iy+1) and the south-east corner of (ix, iy+1).
#include <cooperative_groups.h>
#include <type_traits>
#include <utility>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace sgoc {

static std::atomic<int64_t> g_launches{0};
static inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t kernel_launches() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---- optional per-kernel-class profiler (events pooled and reused) ----
namespace {
struct ProfRec { int kind; cudaEvent_t a, b; double bytes, flops; };
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get() {
    if (used < pool.size()) return pool[used++];
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
    ++used;
    return e;
  }
};
Profiler& prof() { static Profiler p; return p; }
const char* kKindNames[KK_COUNT] = {"sg_operator", "mass", "chebyshev", "mg_smooth", "mg_residual",
                                    "mg_restrict", "mg_prolong", "mg_vcycle_fused", "dot", "minres_scalar",
                                    "vector_update", "mean_exact"};
}  // namespace

const char* kernel_kind_name(int kind) { return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : "?"; }

bool profile_enabled() { return prof().on; }

void profile_enable(bool on) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = on;
  p.recs.clear();
  p.used = 0;
}

ProfScope::ProfScope(int k, cudaStream_t s, double bytes, double flops) : kind(k), st(s), slot(-1) {
  Profiler& p = prof();
  if (!p.on) return;
  std::lock_guard<std::mutex> g(p.mu);
  ProfRec r{k, p.get(), p.get(), bytes, flops};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, s);
  slot = int(p.recs.size());
  p.recs.push_back(r);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  cudaEventRecord(p.recs[slot].b, st);
}

bool profile_query(int kind, int64_t* launches, double* ms, double* bytes, double* flops) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  int64_t nl = 0;
  double t = 0, by = 0, fl = 0;
  for (auto& r : p.recs) {
    if (r.kind != kind) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return false;
    float e = 0;
    if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) return false;
    ++nl; t += e; by += r.bytes; fl += r.flops;
  }
  *launches = nl; *ms = t; *bytes = by; *flops = fl;
  return true;
}

constexpr size_t kMaxSmem = 227 * 1024;   // dynamic shared memory per CTA on sm_103

// Raise a kernel's dynamic shared-memory limit to everything its static shared
// memory leaves.  The limit is a property of the function, not of one launch:
// kept at the maximum, a later and smaller launch never lowers it below what a
// captured (or replayed) launch needs.
template <typename F>
static cudaError_t allow_max_smem(F* f) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxSmem - fa.sharedSizeBytes));
}

// Programmatic dependent launch: every kernel does its work on constant data
// (tables, shared-memory set-up) first, then waits for the grid it depends on
// (griddepcontrol.wait returns once that grid has completed and its memory is
// visible; at once when there is none).  As every kernel waits before it
// touches memory that other kernels write, the stream order of all reads and
// writes is kept, transitively along the chain.  A kernel lets its dependants
// launch (their CTAs then occupy SM resources while they wait) near its end:
// short kernels right after the wait, long ones before their last phase.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_wait(); pdl_trigger(); }

// Streams whose next launch must take a full dependency: the overlap is only
// for a kernel that directly follows another kernel of this library in the same
// stream.  After a cross-stream event wait, a copy or a graph launch the next
// kernel is launched without the attribute (its wait would not cover the work
// on the other stream, which was seen to race).
static std::mutex g_fence_mu;
static std::vector<cudaStream_t> g_fenced;

void pdl_fence(cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_fence_mu);
  for (cudaStream_t s : g_fenced)
    if (s == st) return;
  g_fenced.push_back(st);
}

static bool take_fence(cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_fence_mu);
  for (size_t i = 0; i < g_fenced.size(); ++i)
    if (g_fenced[i] == st) { g_fenced[i] = g_fenced.back(); g_fenced.pop_back(); return true; }
  return false;
}

bool pdl_take_fence(cudaStream_t st) { return take_fence(st); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid; cfg.blockDim = block; cfg.dynamicSmemBytes = smem; cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at; cfg.numAttrs = take_fence(st) ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };

template <typename T>
__device__ __forceinline__ T ldz(const T* __restrict__ X, int ix, int iy, int n1) {
  return (ix >= 0 && ix < n1 && iy >= 0 && iy < n1) ? X[iy * n1 + ix] : T(0);
}

// Sum over the 4 elements of a node of kappa_k(e)/6 * T_e, where
// T_e = 4 X_C - X_a - X_b - 2 X_c (a, b the edge neighbours and c the opposite
// corner of the node inside element e).  Element order: SW, SE, NE, NW.
template <typename T>
__device__ __forceinline__ T dot4(const typename Vec4<T>::type& a, const typename Vec4<T>::type& b) {
  T r = a.x * b.x;
  r = fma(a.y, b.y, r);
  r = fma(a.z, b.z, r);
  r = fma(a.w, b.w, r);
  return r;
}

// ---------------------------------------------------------------------------
// SG operator tile kernel (Sec. 2, Eq. (Zv)): one CTA = TX consecutive nodes
// of one grid row and one slab, all requested chaos columns.
//   phase 0: kappa_k(e)/6 of the 4 elements of each node -> shared
//   phase 1: for every input column alpha, the 4 element terms T_e(alpha) -> shared
//            (and the mass stencil value of the output columns)
//   phase 2: out(beta) = sum_e kappa_0(e) T_e(beta) + sum_{(alpha,k,c)} c sum_e kappa_k(e) T_e(alpha)
// ---------------------------------------------------------------------------
constexpr int kSGThreads = 512;

// asynchronous global->shared copy of one element; invalid elements are zero-filled
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  const int sz = valid ? int(sizeof(T)) : 0;
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// SG operator kernel: one CTA walks rows [r0, r1) of one TX-wide x-tile of one
// slab.  A ring of three X row panels (input columns [in0, in1), TX+2 nodes with
// halo) lives in shared memory; once the element terms of row iy are formed,
// row iy+2 is fetched with cp.async into the slot of row iy-1 while the
// contraction of row iy runs, so every X element is read once per CTA.
//   phase 1: kappa_k(e)/6 of the row's elements; T_e(alpha) for every node and
//            input column (and the mass stencil of the output columns)
//   phase 2: out(beta) = sum_e kappa_0(e) T_e(beta) + sum_{(alpha,k,c)} c sum_e kappa_k(e) T_e(alpha)
// neighbour-table entry staged in shared memory (16 bytes for both types)
template <typename T> struct NbrEntry;
template <> struct __align__(16) NbrEntry<float> { int ts, ks; float c; int pad; };
template <> struct __align__(16) NbrEntry<double> { int ts, ks; double c; };

// Member of a merged SG launch: CTAs of grid z in [g*nslabs, (g+1)*nslabs) work on
// member g, whose operands, coefficient data and scalars replace those of the shared
// arguments (constant indices only, so the member table stays in parameter space).
// Returns the slab index within the member.
template <typename T>
__device__ __forceinline__ int sg_member(SGArgs<T>& a, const SGMulti<T>& m) {
  const int g = int(blockIdx.z) / a.nslabs;
  if (m.ng > 1) {
#pragma unroll
    for (int i = 1; i < kMaxGroup; ++i) {
      if (i == g) {
        a.X = m.X[i]; a.Y = m.Y[i]; a.R = m.R[i]; a.kap = m.kap[i];
        a.c0 = m.c0[i]; a.c1 = m.c1[i]; a.cm = m.cm[i]; a.cr = m.cr[i];
      }
    }
  }
  return int(blockIdx.z) - g * a.nslabs;
}

template <typename T, int TX>
__global__ void __launch_bounds__(kSGThreads, 2) sg_kernel(SGArgs<T> a, const SGMulti<T> mg, int rows_per_cta) {
  const int t = sg_member(a, mg);
  using V4 = typename Vec4<T>::type;
  extern __shared__ __align__(32) unsigned char sg_smem_raw[];
  constexpr int W = TX + 2;
  const int nin = a.in1 - a.in0;
  const int nout = a.out1 - a.out0;
  const bool use_m = a.cm != T(0);
  V4* Ts = reinterpret_cast<V4*>(sg_smem_raw);               // [nin][TX]
  V4* Ks = Ts + size_t(nin) * TX;                            // [M+1][TX]
  T* Ms = reinterpret_cast<T*>(Ks + size_t(a.M + 1) * TX);   // [nout][TX] (when cm != 0)
  T* Xr = Ms + (use_m ? size_t(nout) * TX : 0);              // ring [3][nin][W]
  // the 16-byte table entries start at the next 16-byte boundary after the ring
  const size_t es_off = (size_t(reinterpret_cast<unsigned char*>(Xr + size_t(3) * nin * W) - sg_smem_raw) + 15) &
                        ~size_t(15);
  NbrEntry<T>* Es = reinterpret_cast<NbrEntry<T>*>(sg_smem_raw + es_off);       // [nnz_out]
  int* Ps = reinterpret_cast<int*>(Es + a.nnz_out);          // [nout] first entry of each output column
  int* Pe = Ps + nout;                                       // [nout] end of its entries with k < kmax

  const int ix0 = blockIdx.x * TX;
  const int r0 = blockIdx.y * rows_per_cta;
  const int r1 = min(a.n1, r0 + rows_per_cta);
  const int tid = threadIdx.x;
  const int n1 = a.n1;
  const T* X = a.X + int64_t(t) * a.xs;
  const size_t ring_stride = size_t(nin) * W;

  // neighbour table of the output columns with shared-memory offsets pre-multiplied;
  // per column only the entries with k < kmax (a prefix: the table is sorted by k)
  const int ebase = a.nbr_ptr[a.out0];
  for (int q = tid; q < a.nnz_out; q += kSGThreads) {
    NbrEntry<T> en;
    en.ts = (a.nbr_alpha[ebase + q] - a.in0) * TX;
    en.ks = a.nbr_k[ebase + q] * TX;
    en.c = a.nbr_c[ebase + q];
    Es[q] = en;
  }
  for (int q = tid; q < nout; q += kSGThreads) {
    Ps[q] = a.nbr_ptr[a.out0 + q] - ebase;
    Pe[q] = a.nbr_end[a.out0 + q] - ebase;        // entries with k < kmax (host-computed)
  }

  pdl_wait();                                        // X (and Y, R) are written by earlier kernels
  if (r0 >= r1) { pdl_trigger(); return; }

  // row gy (-1 and n1 give zeros) into ring slot (gy + 1) % 3: a warp per input column,
  // its lanes along the row segment (element lx is grid column ix0 + lx - 1)
  static_assert(W <= 64, "a row segment is at most two lanes' worth per lane");
  const int warp = tid >> 5, lane = tid & 31;
  const int gxa = ix0 + lane - 1, gxb = ix0 + lane + 31;
  const bool seg_a = lane < W, seg_b = lane + 32 < W;
  auto issue_row = [&](int gy) {
    T* dst = Xr + size_t((gy + 1) % 3) * ring_stride;
    const bool rok = gy >= 0 && gy < n1;
    const bool oka = rok && gxa >= 0 && gxa < n1, okb = rok && seg_b && gxb < n1;
    const T* col = X + int64_t(a.in0) * a.n + int64_t(rok ? gy : 0) * n1;
    for (int c = warp; c < nin; c += kSGThreads / 32) {
      const T* cc = col + int64_t(c) * a.n;
      T* dc = dst + c * W;
      if (seg_a) cp_async_elem(dc + lane, oka ? cc + gxa : cc, oka);
      if (seg_b) cp_async_elem(dc + lane + 32, okb ? cc + gxb : cc, okb);
    }
  };
  issue_row(r0 - 1);
  issue_row(r0);
  issue_row(r0 + 1);
  cp_async_commit();

  for (int iy = r0; iy < r1; ++iy) {
    if (iy == r1 - 1) pdl_trigger();
    cp_async_wait<0>();
    __syncthreads();                                   // rows iy-1..iy+1 landed; previous contraction done
    for (int q = tid; q < (a.M + 1) * TX; q += kSGThreads) {
      const int kk = q / TX, lx = q - kk * TX;
      const int ix = min(ix0 + lx, n1 - 1);
      const T* kp = a.kap + int64_t(kk) * a.nx * a.nx;
      V4 v;
      v.x = kp[int64_t(iy) * a.nx + ix];            // SW element (ix, iy)
      v.y = kp[int64_t(iy) * a.nx + ix + 1];        // SE element (ix+1, iy)
      v.z = kp[int64_t(iy + 1) * a.nx + ix + 1];    // NE element (ix+1, iy+1)
      v.w = kp[int64_t(iy + 1) * a.nx + ix];        // NW element (ix, iy+1)
      Ks[kk * TX + lx] = v;
    }
    const T* rS = Xr + size_t(iy % 3) * ring_stride;         // row iy-1
    const T* rC = Xr + size_t((iy + 1) % 3) * ring_stride;   // row iy
    const T* rN = Xr + size_t((iy + 2) % 3) * ring_stride;   // row iy+1
    for (int q = tid; q < nin * TX; q += kSGThreads) {
      const int c = q / TX, lx = q - c * TX;
      const size_t o = size_t(c) * W + lx;
      const T SW = rS[o], S = rS[o + 1], SE = rS[o + 2];
      const T Wv = rC[o], C = rC[o + 1], E = rC[o + 2];
      const T NW = rN[o], N = rN[o + 1], NE = rN[o + 2];
      const T c4 = T(4) * C;
      const T aS = c4 - S, aN = c4 - N;
      V4 v;
      v.x = fma(T(-2), SW, aS - Wv);
      v.y = fma(T(-2), SE, aS - E);
      v.z = fma(T(-2), NE, aN - E);
      v.w = fma(T(-2), NW, aN - Wv);
      Ts[size_t(c) * TX + lx] = v;
      const int col = a.in0 + c;
      if (use_m && col >= a.out0 && col < a.out1) {
        const T edges = (N + S) + (E + Wv);
        const T corners = (NE + NW) + (SE + SW);
        Ms[size_t(col - a.out0) * TX + lx] = a.mass * fma(T(16), C, fma(T(4), edges, corners));
      }
    }
    __syncthreads();                                   // element terms ready; row iy-1 no longer needed
    if (iy + 1 < r1) { issue_row(iy + 2); cp_async_commit(); }
    for (int q = tid; q < nout * TX; q += kSGThreads) {
      const int lx = q % TX, bl = q / TX;
      const int ix = ix0 + lx;
      const int beta = a.out0 + bl;
      T diag = T(0);
      if (!a.no_own) diag = dot4<T>(Ks[lx], Ts[size_t(beta - a.in0) * TX + lx]);
      T off = T(0);
      const int e1 = Pe[bl];
      for (int e = Ps[bl]; e < e1; ++e) {
        const NbrEntry<T> en = Es[e];
        off = fma(en.c, dot4<T>(Ks[en.ks + lx], Ts[en.ts + lx]), off);
      }
      if (ix >= n1) continue;
      T out = fma(a.c0, diag, a.c1 * off);
      if (use_m) out = fma(a.cm, Ms[size_t(bl) * TX + lx], out);
      const int64_t node = int64_t(iy) * n1 + ix;
      if (a.R) out = fma(a.cr, a.R[int64_t(t) * a.rs + int64_t(beta - a.rcol0) * a.n + node], out);
      T* yp = a.Y + int64_t(t) * a.ys + int64_t(beta - a.ycol0) * a.n + node;
      if (a.cy != T(0)) out = fma(a.cy, *yp, out);
      *yp = out;
    }
  }
  cp_async_wait<0>();
}

template <typename T, int TX>
static size_t sg_smem(const SGArgs<T>& a) {
  using V4 = typename Vec4<T>::type;
  const size_t nin = a.in1 - a.in0, nout = a.out1 - a.out0;
  size_t b = sizeof(V4) * (nin * TX + size_t(a.M + 1) * TX) +
             sizeof(T) * ((a.cm != T(0) ? nout * TX : 0) + 3 * nin * (TX + 2));
  b = (b + 15) & ~size_t(15);
  return b + 16 * size_t(a.nnz_out) + sizeof(int) * 2 * nout;
}

template <typename T>
static const SGMulti<T>& sg_solo() {
  static const SGMulti<T> m{};
  return m;
}

template <typename T, int TX>
static cudaError_t launch_sg_tx(const SGArgs<T>& a, size_t smem, cudaStream_t st, const SGMulti<T>& mg) {
  cudaError_t e = allow_max_smem(sg_kernel<T, TX>);
  if (e != cudaSuccess) return e;
  const int xt = (a.n1 + TX - 1) / TX;
  const int per_sm = std::max(1, std::min(2, int((228 * 1024) / (smem + 1024))));
  // about one CTA per resident slot of the GPU: rows per CTA amortise the set-up
  const int64_t want = int64_t(152) * per_sm;
  const int64_t tiles = int64_t(xt) * a.nslabs * mg.ng;
  int rows = int(std::max<int64_t>(1, (tiles * a.n1 + want - 1) / want));
  rows = std::min(rows, a.n1);
  dim3 grid(xt, (a.n1 + rows - 1) / rows, a.nslabs * mg.ng);
  const double w = sizeof(T), cells = double(a.n) * a.nslabs * mg.ng;
  const int nout = a.out1 - a.out0, nin = a.in1 - a.in0;
  const double bytes = w * cells * (nin + nout * (1.0 + (a.R ? 1 : 0) + (a.cy != T(0) ? 1 : 0))) +
                       w * (a.M + 1.0) * a.nx * a.nx;
  const double flops = cells * (15.0 * nin + 9.0 * nout + 9.0 * (a.c1 != T(0) ? a.deg_sum : 0));
  ProfScope ps(KK_SG, st, bytes, flops);
  {
    const cudaError_t le_ = launch_pdl(sg_kernel<T, TX>, dim3(grid), dim3(kSGThreads), size_t(smem), st,
                                      a, mg, rows);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SG apply, quad form: one thread computes four adjacent nodes of one output
// column, so each neighbour-table entry (alpha, k, c) costs eight 4-wide
// shared-memory loads (kappa_k and T_e(alpha) of the four nodes, one plane per
// element) and 20 FMAs for four outputs.  Element terms and kappa are stored
// node-planar ([column][element][node]); the per-node arithmetic and its order
// are those of sg_kernel above.  The output columns are visited in order of
// their entry count (counting sort in the prologue), so the four columns a warp
// works on have about the same trip count.
// ---------------------------------------------------------------------------
constexpr int kSG4Threads = 256;
constexpr int kSG4Bins = 40;          // entry counts per column are <= 2M <= 32

template <typename T, int TX>
static size_t sg4_smem(const SGArgs<T>& a) {
  const size_t nin = a.in1 - a.in0, nout = a.out1 - a.out0;
  size_t b = sizeof(T) * (nin * 4 * TX + 2 * size_t(a.M + 1) * 4 * TX + (a.cm != T(0) ? nout * TX : 0) +
                          3 * nin * (TX + 2));
  b = (b + 15) & ~size_t(15);
  return b + 16 * size_t(a.nnz_out) + sizeof(int) * (3 * nout + 2 * kSG4Bins);
}

template <typename T, int TX, int MINB>
__global__ void __launch_bounds__(kSG4Threads, MINB) sg4_kernel(SGArgs<T> a, const SGMulti<T> mg, int rows_per_cta) {
  const int t = sg_member(a, mg);
  using V4 = typename Vec4<T>::type;
  constexpr int NQ = TX / 4;          // quads per row of the tile
  constexpr int W = TX + 2;
  constexpr int NT = kSG4Threads;
  extern __shared__ __align__(32) unsigned char sg_smem_raw[];
  const int nin = a.in1 - a.in0;
  const int nout = a.out1 - a.out0;
  const bool use_m = a.cm != T(0);
  T* Ts = reinterpret_cast<T*>(sg_smem_raw);                 // [nin][4][TX]
  T* Ks = Ts + size_t(nin) * 4 * TX;                         // [2][M+1][4][TX]: rows of alternating parity
  const size_t kslot = size_t(a.M + 1) * 4 * TX;
  T* Ms = Ks + 2 * kslot;                                    // [nout][TX] (when cm != 0)
  T* Xr = Ms + (use_m ? size_t(nout) * TX : 0);              // ring [3][nin][W]
  const size_t es_off = (size_t(reinterpret_cast<unsigned char*>(Xr + size_t(3) * nin * W) - sg_smem_raw) + 15) &
                        ~size_t(15);
  NbrEntry<T>* Es = reinterpret_cast<NbrEntry<T>*>(sg_smem_raw + es_off);       // [nnz_out]
  int* Ps = reinterpret_cast<int*>(Es + a.nnz_out);          // [nout]
  int* Pe = Ps + nout;                                       // [nout]
  int* Ord = Pe + nout;                                      // [nout] output columns by entry count
  int* Hist = Ord + nout;                                    // [2][kSG4Bins]
  const V4* Ts4 = reinterpret_cast<const V4*>(Ts);

  const int ix0 = blockIdx.x * TX;
  const int r0 = blockIdx.y * rows_per_cta;
  const int r1 = min(a.n1, r0 + rows_per_cta);
  const int tid = threadIdx.x;
  const int n1 = a.n1;
  const T* X = a.X + int64_t(t) * a.xs;
  const size_t ring_stride = size_t(nin) * W;

  // neighbour table of the output columns (offsets in 4-node units) and the visiting order
  const int ebase = a.nbr_ptr[a.out0];
  for (int q = tid; q < a.nnz_out; q += NT) {
    NbrEntry<T> en;
    en.ts = (a.nbr_alpha[ebase + q] - a.in0) * TX;
    en.ks = a.nbr_k[ebase + q] * TX;
    en.c = a.nbr_c[ebase + q];
    Es[q] = en;
  }
  for (int q = tid; q < kSG4Bins; q += NT) Hist[q] = 0;
  __syncthreads();
  for (int q = tid; q < nout; q += NT) {
    const int p0 = a.nbr_ptr[a.out0 + q] - ebase, p1 = a.nbr_end[a.out0 + q] - ebase;
    Ps[q] = p0;
    Pe[q] = p1;
    atomicAdd(&Hist[min(p1 - p0, kSG4Bins - 1)], 1);
  }
  __syncthreads();
  if (tid == 0) {                                    // start of each count class, longest first
    int acc = 0;
    for (int b = kSG4Bins - 1; b >= 0; --b) { const int h = Hist[b]; Hist[b] = acc; acc += h; }
  }
  __syncthreads();
  for (int q = tid; q < nout; q += NT) Ord[atomicAdd(&Hist[min(Pe[q] - Ps[q], kSG4Bins - 1)], 1)] = q;

  pdl_wait();                                        // X (and Y, R) are written by earlier kernels
  if (r0 >= r1) { pdl_trigger(); return; }

  // row gy (-1 and n1 give zeros) into ring slot (gy + 1) % 3: a warp per input column,
  // its lanes along the row segment (element lx is grid column ix0 + lx - 1)
  static_assert(W <= 64, "a row segment is at most two lanes' worth per lane");
  const int warp = tid >> 5, lane = tid & 31;
  const int gxa = ix0 + lane - 1, gxb = ix0 + lane + 31;
  const bool seg_a = lane < W, seg_b = lane + 32 < W;
  auto issue_row = [&](int gy) {
    T* dst = Xr + size_t((gy + 1) % 3) * ring_stride;
    const bool rok = gy >= 0 && gy < n1;
    const bool oka = rok && gxa >= 0 && gxa < n1, okb = rok && seg_b && gxb < n1;
    const T* col = X + int64_t(a.in0) * a.n + int64_t(rok ? gy : 0) * n1;
    T* d = dst;
    for (int c = warp; c < nin; c += NT / 32) {
      const T* cc = col + int64_t(c) * a.n;
      T* dc = d + c * W;
      if (seg_a) cp_async_elem(dc + lane, oka ? cc + gxa : cc, oka);
      if (seg_b) cp_async_elem(dc + lane + 32, okb ? cc + gxb : cc, okb);
    }
  };
  // kappa_k/6 of the four elements of every node of row gy (SW, SE, NE, NW planes) into slot
  // gy & 1: a warp per (k, element) plane, its lanes along the tile
  auto issue_kappa = [&](int gy) {
    T* dst = Ks + size_t(gy & 1) * kslot;
    for (int pl = warp; pl < (a.M + 1) * 4; pl += NT / 32) {
      const int kk = pl >> 2, e = pl & 3;
      const int ey = gy + (e >= 2 ? 1 : 0);
      const T* kp = a.kap + (int64_t(kk) * a.nx + ey) * a.nx + ((e == 1 || e == 2) ? 1 : 0);
      for (int lx = lane; lx < TX; lx += 32)
        cp_async_elem(dst + size_t(pl) * TX + lx, kp + min(ix0 + lx, n1 - 1), true);
    }
  };
  issue_row(r0 - 1);
  issue_row(r0);
  issue_row(r0 + 1);
  issue_kappa(r0);
  cp_async_commit();

  for (int iy = r0; iy < r1; ++iy) {
    if (iy == r1 - 1) pdl_trigger();
    cp_async_wait<0>();
    __syncthreads();                                   // rows iy-1..iy+1 and kappa landed; previous contraction done
    const V4* Ks4 = reinterpret_cast<const V4*>(Ks + size_t(iy & 1) * kslot);
    const T* rS = Xr + size_t(iy % 3) * ring_stride;         // row iy-1
    const T* rC = Xr + size_t((iy + 1) % 3) * ring_stride;   // row iy
    const T* rN = Xr + size_t((iy + 2) % 3) * ring_stride;   // row iy+1
    // element terms T_e(alpha) of four nodes per item
    for (int q = tid; q < nin * NQ; q += NT) {
      const int c = q / NQ, qd = q - c * NQ;
      const size_t o = size_t(c) * W + 4 * qd;
      T s[6], m[6], nn[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) { s[j] = rS[o + j]; m[j] = rC[o + j]; nn[j] = rN[o + j]; }
      T tv[4][4];                                     // [element][node]
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T SW = s[u], S = s[u + 1], SE = s[u + 2];
        const T Wv = m[u], C = m[u + 1], E = m[u + 2];
        const T NW = nn[u], N = nn[u + 1], NE = nn[u + 2];
        const T c4 = T(4) * C;
        const T aS = c4 - S, aN = c4 - N;
        tv[0][u] = fma(T(-2), SW, aS - Wv);
        tv[1][u] = fma(T(-2), SE, aS - E);
        tv[2][u] = fma(T(-2), NE, aN - E);
        tv[3][u] = fma(T(-2), NW, aN - Wv);
      }
      V4* dst = reinterpret_cast<V4*>(Ts) + size_t(c) * 4 * NQ + qd;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        V4 v; v.x = tv[e][0]; v.y = tv[e][1]; v.z = tv[e][2]; v.w = tv[e][3];
        dst[e * NQ] = v;
      }
      const int col = a.in0 + c;
      if (use_m && col >= a.out0 && col < a.out1) {
        V4 mv;
        T* mp = &mv.x;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T edges = (nn[u + 1] + s[u + 1]) + (m[u + 2] + m[u]);
          const T corners = (nn[u + 2] + nn[u]) + (s[u + 2] + s[u]);
          mp[u] = a.mass * fma(T(16), m[u + 1], fma(T(4), edges, corners));
        }
        reinterpret_cast<V4*>(Ms)[size_t(col - a.out0) * NQ + qd] = mv;
      }
    }
    __syncthreads();                                   // element terms ready; row iy-1 no longer needed
    if (iy + 1 < r1) { issue_row(iy + 2); issue_kappa(iy + 1); cp_async_commit(); }
    for (int q = tid; q < nout * NQ; q += NT) {
      const int sl = q / NQ, qd = q - sl * NQ;
      const int bl = Ord[sl];
      const int beta = a.out0 + bl;
      T diag[4] = {T(0), T(0), T(0), T(0)}, off[4];
      if (!a.no_own) {
        const V4* kb = Ks4 + qd;
        const V4* tb = Ts4 + size_t(beta - a.in0) * TX + qd;
        const V4 k0 = kb[0], k1 = kb[NQ], k2 = kb[2 * NQ], k3 = kb[3 * NQ];
        const V4 t0 = tb[0], t1 = tb[NQ], t2 = tb[2 * NQ], t3 = tb[3 * NQ];
        diag[0] = fma(k3.x, t3.x, fma(k2.x, t2.x, fma(k1.x, t1.x, k0.x * t0.x)));
        diag[1] = fma(k3.y, t3.y, fma(k2.y, t2.y, fma(k1.y, t1.y, k0.y * t0.y)));
        diag[2] = fma(k3.z, t3.z, fma(k2.z, t2.z, fma(k1.z, t1.z, k0.z * t0.z)));
        diag[3] = fma(k3.w, t3.w, fma(k2.w, t2.w, fma(k1.w, t1.w, k0.w * t0.w)));
      }
      off[0] = off[1] = off[2] = off[3] = T(0);
      const int e1 = Pe[bl];
      for (int e = Ps[bl]; e < e1; ++e) {
        const NbrEntry<T> en = Es[e];
        const V4* kb = Ks4 + en.ks + qd;
        const V4* tb = Ts4 + en.ts + qd;
        const V4 k0 = kb[0], k1 = kb[NQ], k2 = kb[2 * NQ], k3 = kb[3 * NQ];
        const V4 t0 = tb[0], t1 = tb[NQ], t2 = tb[2 * NQ], t3 = tb[3 * NQ];
        off[0] = fma(en.c, fma(k3.x, t3.x, fma(k2.x, t2.x, fma(k1.x, t1.x, k0.x * t0.x))), off[0]);
        off[1] = fma(en.c, fma(k3.y, t3.y, fma(k2.y, t2.y, fma(k1.y, t1.y, k0.y * t0.y))), off[1]);
        off[2] = fma(en.c, fma(k3.z, t3.z, fma(k2.z, t2.z, fma(k1.z, t1.z, k0.z * t0.z))), off[2]);
        off[3] = fma(en.c, fma(k3.w, t3.w, fma(k2.w, t2.w, fma(k1.w, t1.w, k0.w * t0.w))), off[3]);
      }
      const T* mrow = use_m ? Ms + size_t(bl) * TX + 4 * qd : nullptr;
      const int64_t rowbase = int64_t(iy) * n1;
      T* ycol = a.Y + int64_t(t) * a.ys + int64_t(beta - a.ycol0) * a.n;
      const T* rcol = a.R ? a.R + int64_t(t) * a.rs + int64_t(beta - a.rcol0) * a.n : nullptr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ix = ix0 + 4 * qd + u;
        if (ix >= n1) break;
        T out = fma(a.c0, diag[u], a.c1 * off[u]);
        if (use_m) out = fma(a.cm, mrow[u], out);
        const int64_t node = rowbase + ix;
        if (rcol) out = fma(a.cr, rcol[node], out);
        T* yp = ycol + node;
        if (a.cy != T(0)) out = fma(a.cy, *yp, out);
        *yp = out;
      }
    }
  }
  cp_async_wait<0>();
}

template <typename T, int TX, int MINB>
static cudaError_t launch_sg4_tx(const SGArgs<T>& a, size_t smem, cudaStream_t st, const SGMulti<T>& mg) {
  cudaError_t e = allow_max_smem(sg4_kernel<T, TX, MINB>);
  if (e != cudaSuccess) return e;
  const int xt = (a.n1 + TX - 1) / TX;
  // resident CTAs per SM: shared memory, and registers (launch bounds: MINB of 256 threads)
  const int per_sm = std::max(1, std::min(MINB, int((228 * 1024) / (smem + 1024))));
  const int64_t want = int64_t(152) * per_sm;
  const int64_t tiles = int64_t(xt) * a.nslabs * mg.ng;
  int rows = int(std::max<int64_t>(1, (tiles * a.n1 + want - 1) / want));
  rows = std::min(rows, a.n1);
  dim3 grid(xt, (a.n1 + rows - 1) / rows, a.nslabs * mg.ng);
  const double w = sizeof(T), cells = double(a.n) * a.nslabs * mg.ng;
  const int nout = a.out1 - a.out0, nin = a.in1 - a.in0;
  const double bytes = w * cells * (nin + nout * (1.0 + (a.R ? 1 : 0) + (a.cy != T(0) ? 1 : 0))) +
                       w * (a.M + 1.0) * a.nx * a.nx;
  const double flops = cells * (15.0 * nin + 9.0 * nout + 9.0 * (a.c1 != T(0) ? a.deg_sum : 0));
  ProfScope ps(KK_SG, st, bytes, flops);
  {
    const cudaError_t le_ = launch_pdl(sg4_kernel<T, TX, MINB>, dim3(grid), dim3(kSG4Threads), size_t(smem), st,
                                      a, mg, rows);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SG apply, two-phase form (float32): per row of a 32-node tile,
//   phase 1: a warp takes one input column alpha (lane = node), forms the element
//            terms T_e(alpha) from the staged rows and, with kappa_k of its node in
//            registers, writes U_k(alpha) = sum_e kappa_k(e) T_e(alpha) for exactly
//            the k the shape's outputs use (slot table, bit k of the column's mask);
//   phase 2: a warp takes one output column beta and gathers
//            out = c0 U_0(beta) + c1 sum_entries c U_k(alpha) from the slot list.
// Every shared-memory access is lane-consecutive (no bank conflicts) and moves
// 4 bytes per node and product, against 32 for the quad form.  Products and
// sums are formed in the same order as in sg_kernel.
// ---------------------------------------------------------------------------
constexpr int kSGUThreads = 512;

__host__ __device__ __forceinline__ size_t align8(size_t b) { return (b + 7) & ~size_t(7); }

static size_t sgu_smem(const SGArgs<float>& a) {
  const size_t nin = a.in1 - a.in0, nout = a.out1 - a.out0;
  size_t b = 4 * (3 * nin * 34 + size_t(a.u_nslots) * 32 + (a.cm != 0.f ? nout * 32 : 0) + 2 * size_t(a.M + 1) * 4 * 32);
  b = align8(b) + 8 * nin + 4 * nout + 4 * (nout + 1);
  return align8(b) + 8 * size_t(a.u_nent);
}

template <int KM>
__global__ void __launch_bounds__(kSGUThreads, 1) sgu_kernel(SGArgs<float> a, const SGMulti<float> mg, int rows_per_cta) {
  const int t = sg_member(a, mg);
  constexpr int TX = 32, W = TX + 2, NW = kSGUThreads / 32;
  extern __shared__ __align__(16) unsigned char sgu_smem_raw[];
  const int nin = a.in1 - a.in0;
  const int nout = a.out1 - a.out0;
  const bool use_m = a.cm != 0.f;
  float* Xr = reinterpret_cast<float*>(sgu_smem_raw);                 // ring [3][nin][W]
  float* U = Xr + size_t(3) * nin * W;                                 // [nslots][TX]
  float* Ms = U + size_t(a.u_nslots) * TX;                             // [nout][TX] when cm != 0
  float* Ks = Ms + (use_m ? size_t(nout) * TX : 0);                    // [2][M+1][4][TX] by row parity
  const int kslot = (a.M + 1) * 4 * TX;
  unsigned char* tail = reinterpret_cast<unsigned char*>(Ks + 2 * size_t(kslot));
  int2* MB = reinterpret_cast<int2*>(sgu_smem_raw + align8(size_t(tail - sgu_smem_raw)));   // [nin]
  int* Dg = reinterpret_cast<int*>(MB + nin);                          // [nout]
  int* Ep = Dg + nout;                                                 // [nout + 1]
  int2* Et = reinterpret_cast<int2*>(sgu_smem_raw + align8(size_t(reinterpret_cast<unsigned char*>(Ep + nout + 1) -
                                                                  sgu_smem_raw)));                  // [nent]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ix0 = blockIdx.x * TX;
  const int r0 = blockIdx.y * rows_per_cta;
  const int r1 = min(a.n1, r0 + rows_per_cta);
  const int n1 = a.n1;
  const float* X = a.X + int64_t(t) * a.xs;
  const size_t ring_stride = size_t(nin) * W;

  // slot table of the shape (constant data)
  const int2* mbg = reinterpret_cast<const int2*>(a.u_mb);
  for (int q = tid; q < nin; q += kSGUThreads) MB[q] = mbg[q];
  for (int q = tid; q < nout; q += kSGUThreads) Dg[q] = a.u_diag[q];
  for (int q = tid; q <= nout; q += kSGUThreads) Ep[q] = a.u_eptr[q];
  for (int q = tid; q < a.u_nent; q += kSGUThreads) Et[q] = a.u_e32[q];

  pdl_wait();                                        // X (and Y, R) are written by earlier kernels
  if (r0 >= r1) { pdl_trigger(); return; }

  // ring row gy: one warp per input column, lanes along x (34 values: lanes 0..31, then 0..1)
  auto issue_row = [&](int gy) {
    float* dst = Xr + size_t((gy + 1) % 3) * ring_stride;
    const bool rok = gy >= 0 && gy < n1;
    const int gx0 = ix0 + lane - 1, gx1 = ix0 + lane + 31;
    const bool ok0 = rok && gx0 >= 0 && gx0 < n1, ok1 = rok && lane < 2 && gx1 < n1;
    const float* src = X + int64_t(a.in0 + warp) * a.n + int64_t(rok ? gy : 0) * n1;
    float* d = dst + size_t(warp) * W + lane;
    for (int c = warp; c < nin; c += NW) {
      cp_async_elem(d, ok0 ? src + gx0 : src, ok0);
      if (lane < 2) cp_async_elem(d + 32, ok1 ? src + gx1 : src, ok1);
      src += int64_t(NW) * a.n;
      d += size_t(NW) * W;
    }
  };
  // kappa_k/6 of the four elements of every node of row gy (SW, SE, NE, NW planes) into slot gy & 1
  const int nxk = a.nx;
  auto issue_kappa = [&](int gy) {
    float* dst = Ks + (gy & 1) * kslot;
    for (int q = tid; q < kslot; q += kSGUThreads) {
      const int kk = q >> 7, r = q & 127;              // 4 * TX = 128 values per k
      const int e = r >> 5, lx = r & 31;
      const int ix = min(ix0 + lx, n1 - 1);
      const int ex = ix + ((e == 1 || e == 2) ? 1 : 0), ey = gy + (e >= 2 ? 1 : 0);
      cp_async_elem(dst + q, a.kap + (int64_t(kk) * nxk + ey) * nxk + ex, true);
    }
  };
  issue_row(r0 - 1);
  issue_row(r0);
  issue_row(r0 + 1);
  issue_kappa(r0);
  cp_async_commit();

  for (int iy = r0; iy < r1; ++iy) {
    if (iy == r1 - 1) pdl_trigger();
    cp_async_wait<0>();
    __syncthreads();                                   // rows iy-1..iy+1 and kappa landed; previous gathers done
    const float* Kr = Ks + (iy & 1) * kslot;
    float kr[KM][4];
#pragma unroll
    for (int k = 0; k < KM; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) kr[k][e] = k <= a.M ? Kr[(k * 4 + e) * TX + lane] : 0.f;
    const float* rS = Xr + size_t(iy % 3) * ring_stride;         // row iy-1
    const float* rC = Xr + size_t((iy + 1) % 3) * ring_stride;   // row iy
    const float* rN = Xr + size_t((iy + 2) % 3) * ring_stride;   // row iy+1
    for (int c = warp; c < nin; c += NW) {
      const size_t o = size_t(c) * W + lane;
      const float SW = rS[o], S = rS[o + 1], SE = rS[o + 2];
      const float Wv = rC[o], C = rC[o + 1], E = rC[o + 2];
      const float NW_ = rN[o], N = rN[o + 1], NE = rN[o + 2];
      const float c4 = 4.f * C;
      const float aS = c4 - S, aN = c4 - N;
      const float T0 = fmaf(-2.f, SW, aS - Wv);
      const float T1 = fmaf(-2.f, SE, aS - E);
      const float T2 = fmaf(-2.f, NE, aN - E);
      const float T3 = fmaf(-2.f, NW_, aN - Wv);
      const int2 mb = MB[c];
      const unsigned mask = unsigned(mb.x);
      float* up = U + size_t(mb.y) * TX + lane;
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        if (mask & (1u << k)) {
          float d = kr[k][0] * T0;
          d = fmaf(kr[k][1], T1, d);
          d = fmaf(kr[k][2], T2, d);
          d = fmaf(kr[k][3], T3, d);
          *up = d;
          up += TX;
        }
      }
      const int col = a.in0 + c;
      if (use_m && col >= a.out0 && col < a.out1) {
        const float edges = (N + S) + (E + Wv);
        const float corners = (NE + NW_) + (SE + SW);
        Ms[size_t(col - a.out0) * TX + lane] = a.mass * fmaf(16.f, C, fmaf(4.f, edges, corners));
      }
    }
    __syncthreads();                                   // products ready; row iy-1 no longer needed
    if (iy + 1 < r1) { issue_row(iy + 2); issue_kappa(iy + 1); cp_async_commit(); }
    const int ix = ix0 + lane;
    for (int bl = warp; bl < nout; bl += NW) {
      const int beta = a.out0 + bl;
      const float* ul = U + lane;
      const float diag = a.no_own ? 0.f : ul[Dg[bl] * TX];
      float off = 0.f;
      const int e1 = Ep[bl + 1];
      for (int e = Ep[bl]; e < e1; ++e) {
        const int2 en = Et[e];                         // (slot * 32, bits of c)
        off = fmaf(__int_as_float(en.y), ul[en.x], off);
      }
      if (ix >= n1) continue;
      float out = fmaf(a.c0, diag, a.c1 * off);
      if (use_m) out = fmaf(a.cm, Ms[size_t(bl) * TX + lane], out);
      const int64_t node = int64_t(iy) * n1 + ix;
      if (a.R) out = fmaf(a.cr, a.R[int64_t(t) * a.rs + int64_t(beta - a.rcol0) * a.n + node], out);
      float* yp = a.Y + int64_t(t) * a.ys + int64_t(beta - a.ycol0) * a.n + node;
      if (a.cy != 0.f) out = fmaf(a.cy, *yp, out);
      *yp = out;
    }
  }
  cp_async_wait<0>();
}

template <int KM>
static cudaError_t launch_sgu_km(const SGArgs<float>& a, size_t smem, cudaStream_t st, const SGMulti<float>& mg) {
  cudaError_t e = allow_max_smem(sgu_kernel<KM>);
  if (e != cudaSuccess) return e;
  constexpr int TX = 32;
  const int xt = (a.n1 + TX - 1) / TX;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sgu_kernel<KM>, kSGUThreads, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, per_sm);
  const int64_t want = int64_t(152) * per_sm;
  const int64_t tiles = int64_t(xt) * a.nslabs * mg.ng;
  int rows = int(std::max<int64_t>(1, (tiles * a.n1 + want - 1) / want));
  rows = std::min(rows, a.n1);
  dim3 grid(xt, (a.n1 + rows - 1) / rows, a.nslabs * mg.ng);
  const double w = 4.0, cells = double(a.n) * a.nslabs * mg.ng;
  const int nout = a.out1 - a.out0, nin = a.in1 - a.in0;
  const double bytes = w * cells * (nin + nout * (1.0 + (a.R ? 1 : 0) + (a.cy != 0.f ? 1 : 0))) +
                       w * (a.M + 1.0) * a.nx * a.nx;
  const double flops = cells * (15.0 * nin + 9.0 * nout + 9.0 * (a.c1 != 0.f ? a.deg_sum : 0));
  ProfScope ps(KK_SG, st, bytes, flops);
  {
    const cudaError_t le_ = launch_pdl(sgu_kernel<KM>, dim3(grid), dim3(kSGUThreads), size_t(smem), st, a, mg, rows);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// the two-phase kernel when the shape has a slot table that fits in shared memory
static bool try_launch_sgu(const SGArgs<float>& a, cudaStream_t st, cudaError_t* err, const SGMulti<float>& mg) {
  if (!a.u_mb || a.n1 < 24 || a.M + 1 > 17) return false;
  const size_t smem = sgu_smem(a);
  if (smem + 4096 > kMaxSmem) return false;
  if (a.M + 1 <= 5) *err = launch_sgu_km<5>(a, smem, st, mg);
  else if (a.M + 1 <= 9) *err = launch_sgu_km<9>(a, smem, st, mg);
  else *err = launch_sgu_km<17>(a, smem, st, mg);
  return true;
}

// ---------------------------------------------------------------------------
// SG apply, direct form: one thread per (node, output column), no shared memory
// and no barriers; each element term is formed from its column's 3 x 3
// neighbourhood read through the cache, once per table entry that needs it.  For
// launch shapes with few output columns and few couplings (the hGS visits of the
// low chaos levels), where the staged forms' fixed costs (table and kappa staging,
// row pipelines) dominate.  The per-node arithmetic and its order are those of
// sg_kernel.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) sgd_kernel(SGArgs<T> a, const SGMulti<T> mg) {
  const int t = sg_member(a, mg);
  using V4 = typename Vec4<T>::type;
  const int64_t node = int64_t(blockIdx.x) * 256 + threadIdx.x;
  const int beta = a.out0 + int(blockIdx.y);
  const int n1 = a.n1;
  const bool live = node < a.n;
  const int iy = live ? int(node / n1) : 0, ix = live ? int(node - int64_t(iy) * n1) : 0;
  const int64_t nx = a.nx;
  const int e0 = a.nbr_ptr[beta], e1 = a.nbr_end[beta];
  pdl_enter();                                       // X, R and Y are written by earlier kernels
  if (!live) return;
  const T* X = a.X + int64_t(t) * a.xs;
  const bool use_m = a.cm != T(0);
  const bool xl = ix > 0, xr = ix + 1 < n1, yd = iy > 0, yu = iy + 1 < n1;
  // the 3 x 3 neighbourhood of column col (zero outside the grid) and its element terms
  auto nb9 = [&](int col, T (&v)[9]) {
    const T* c = X + int64_t(col) * a.n + node;
    v[0] = (yd && xl) ? c[-n1 - 1] : T(0); v[1] = yd ? c[-n1] : T(0); v[2] = (yd && xr) ? c[-n1 + 1] : T(0);
    v[3] = xl ? c[-1] : T(0);              v[4] = c[0];               v[5] = xr ? c[1] : T(0);
    v[6] = (yu && xl) ? c[n1 - 1] : T(0);  v[7] = yu ? c[n1] : T(0);  v[8] = (yu && xr) ? c[n1 + 1] : T(0);
  };
  auto terms = [&](const T (&v)[9]) {
    const T SW = v[0], S = v[1], SE = v[2], Wv = v[3], C = v[4], E = v[5], NW = v[6], N = v[7], NE = v[8];
    const T c4 = T(4) * C;
    const T aS = c4 - S, aN = c4 - N;
    V4 r;
    r.x = fma(T(-2), SW, aS - Wv);
    r.y = fma(T(-2), SE, aS - E);
    r.z = fma(T(-2), NE, aN - E);
    r.w = fma(T(-2), NW, aN - Wv);
    return r;
  };
  auto kap4 = [&](int k) {
    const T* kp = a.kap + int64_t(k) * nx * nx;
    V4 r;
    r.x = kp[int64_t(iy) * nx + ix];             // SW element (ix, iy)
    r.y = kp[int64_t(iy) * nx + ix + 1];         // SE element (ix+1, iy)
    r.z = kp[int64_t(iy + 1) * nx + ix + 1];     // NE element (ix+1, iy+1)
    r.w = kp[int64_t(iy + 1) * nx + ix];         // NW element (ix, iy+1)
    return r;
  };
  T diag = T(0), mass = T(0);
  if (!a.no_own || use_m) {
    T v[9];
    nb9(beta, v);
    if (!a.no_own) diag = dot4<T>(kap4(0), terms(v));
    if (use_m) {
      const T edges = (v[7] + v[1]) + (v[5] + v[3]);
      const T corners = (v[8] + v[6]) + (v[2] + v[0]);
      mass = a.mass * fma(T(16), v[4], fma(T(4), edges, corners));
    }
  }
  T off = T(0);
  for (int e = e0; e < e1; ++e) {
    T v[9];
    nb9(a.nbr_alpha[e], v);
    off = fma(a.nbr_c[e], dot4<T>(kap4(a.nbr_k[e]), terms(v)), off);
  }
  T out = fma(a.c0, diag, a.c1 * off);
  if (use_m) out = fma(a.cm, mass, out);
  if (a.R) out = fma(a.cr, a.R[int64_t(t) * a.rs + int64_t(beta - a.rcol0) * a.n + node], out);
  T* yp = a.Y + int64_t(t) * a.ys + int64_t(beta - a.ycol0) * a.n + node;
  if (a.cy != T(0)) out = fma(a.cy, *yp, out);
  *yp = out;
}

template <typename T>
static cudaError_t launch_sgd(const SGArgs<T>& a, cudaStream_t st, const SGMulti<T>& mg) {
  const int nout = a.out1 - a.out0;
  dim3 grid(unsigned((a.n + 255) / 256), unsigned(nout), unsigned(a.nslabs * mg.ng));
  const double w = sizeof(T), cells = double(a.n) * a.nslabs * mg.ng;
  const double bytes = w * cells * (double(a.in1 - a.in0) + nout * (1.0 + (a.R ? 1 : 0) + (a.cy != T(0) ? 1 : 0))) +
                       w * (a.M + 1.0) * a.nx * a.nx;
  const double flops = cells * (15.0 * (nout + (a.c1 != T(0) ? a.deg_sum : 0)) + 9.0 * nout +
                                9.0 * (a.c1 != T(0) ? a.deg_sum : 0));
  ProfScope ps(KK_SG, st, bytes, flops);
  {
    const cudaError_t le_ = launch_pdl(sgd_kernel<T>, grid, dim3(256), size_t(0), st, a, mg);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SG apply, register form (variant 7; float32, Legendre chaos of a compiled (M, p)).
// One thread per node keeps the coupling sum of every chaos column in registers and
// reads each input column once: from the 3 x 3 neighbourhood of X(alpha) (a 32 x 4
// node tile with its halo, staged in shared memory) it forms the element terms
// T_e(alpha), the diagonal term sum_e kappa_0(e) T_e(alpha) and the mass stencil when
// alpha is an output column (kept in shared memory for the epilogue), and for every
// kept k the product U_k(alpha) = sum_e kappa_k(e) T_e(alpha), added with its
// coefficient to the outputs alpha + e_k and alpha - e_k.  The multi-indices and
// their neighbours are a compile-time table, so every register index is a constant.
// The products and the epilogue are those of the other variants; a column's coupling
// terms arrive in increasing alpha rather than increasing k (agreement to rounding).
// ---------------------------------------------------------------------------
constexpr int binom_c(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return int(r);
}
// compositions of s into `parts` nonnegative parts
constexpr int ncomp_c(int s, int parts) { return parts == 0 ? (s == 0 ? 1 : 0) : binom_c(s + parts - 1, parts - 1); }

// graded multi-indices of total degree <= PD, lexicographically descending within a degree
// (the order of the problem set-up, checked against it at launch), and their neighbours
template <int M, int PD>
struct LegChaos {
  static constexpr int P = binom_c(M + PD, PD);
  int idx[P][M];
  int up[P][M];    // index of alpha + e_k, -1 beyond degree PD
  int dn[P][M];    // index of alpha - e_k, -1 when alpha_k = 0
  static constexpr int index_of(const int (&b)[M]) {
    int deg = 0;
    for (int j = 0; j < M; ++j) deg += b[j];
    int r = binom_c(M + deg - 1, M);          // multi-indices of lower degree
    int rem = deg;
    for (int i = 0; i + 1 < M; ++i) {         // lexicographically greater ones of this degree
      for (int v = b[i] + 1; v <= rem; ++v) r += ncomp_c(rem - v, M - i - 1);
      rem -= b[i];
    }
    return r;
  }
  constexpr LegChaos() : idx(), up(), dn() {
    int a[M] = {};
    int pos = 0;
    for (int deg = 0; deg <= PD; ++deg) {
      for (int j = 0; j < M; ++j) a[j] = 0;
      a[0] = deg;
      while (true) {
        for (int j = 0; j < M; ++j) idx[pos][j] = a[j];
        ++pos;
        int i = M - 2;                        // next smaller composition of deg
        while (i >= 0 && a[i] == 0) --i;
        if (i < 0) break;
        int tail = 0;
        for (int j = i + 1; j < M; ++j) { tail += a[j]; a[j] = 0; }
        a[i] -= 1;
        a[i + 1] = tail + 1;
      }
    }
    for (int q = 0; q < P; ++q) {
      int deg = 0;
      for (int j = 0; j < M; ++j) deg += idx[q][j];
      for (int k = 0; k < M; ++k) {
        int b[M] = {};
        for (int j = 0; j < M; ++j) b[j] = idx[q][j];
        b[k] += 1;
        up[q][k] = deg < PD ? index_of(b) : -1;
        b[k] -= 2;
        dn[q][k] = idx[q][k] > 0 ? index_of(b) : -1;
      }
    }
  }
};
template <int M, int PD>
struct LegTab {
  static constexpr LegChaos<M, PD> t{};
};

constexpr int kSGRTX = 32, kSGRTY = 4, kSGRThreads = kSGRTX * kSGRTY;

template <int... Is, typename F>
__device__ __forceinline__ void static_for(std::integer_sequence<int, Is...>, F&& f) {
  (f(std::integral_constant<int, Is>{}), ...);
}

inline size_t sgr_smem(int nin, int nout, bool own, bool use_m) {
  return sizeof(float) * (size_t(nin) * (kSGRTY + 2) * (kSGRTX + 2) +
                          size_t(nout) * kSGRThreads * ((own ? 1 : 0) + (use_m ? 1 : 0)));
}

template <int M, int PD>
__global__ void __launch_bounds__(kSGRThreads, 1) sgr_kernel(SGArgs<float> a, const SGMulti<float> mg) {
  using Tab = LegTab<M, PD>;
  constexpr int P = LegChaos<M, PD>::P;
  constexpr int WX = kSGRTX + 2, WY = kSGRTY + 2, TS = WX * WY;
  const int t = sg_member(a, mg);
  extern __shared__ __align__(16) float sgr_smem_f[];
  const int nin = a.in1 - a.in0, nout = a.out1 - a.out0;
  const bool own = !a.no_own, use_m = a.cm != 0.0f;
  float* Xs = sgr_smem_f;                                    // [nin][WY][WX]
  float* Ds = Xs + size_t(nin) * TS;                         // [nout][threads] diagonal terms
  float* Ms = Ds + (own ? size_t(nout) * kSGRThreads : 0);   // [nout][threads] mass terms
  const int tx = threadIdx.x % kSGRTX, ty = threadIdx.x / kSGRTX;
  const int ix0 = blockIdx.x * kSGRTX, iy0 = blockIdx.y * kSGRTY;
  const int n1 = a.n1, ix = ix0 + tx, iy = iy0 + ty;
  const bool live = ix < n1 && iy < n1;
  // kappa_k(e)/6 of the node's four elements (SW, SE, NE, NW), clamped at the edge
  float kk[M + 1][4];
  {
    const int cx = min(ix, n1 - 1), cy = min(iy, n1 - 1);
#pragma unroll
    for (int k = 0; k <= M; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ex = cx + ((e == 1 || e == 2) ? 1 : 0), ey = cy + (e >= 2 ? 1 : 0);
        kk[k][e] = a.kap[(int64_t(k) * a.nx + ey) * a.nx + ex];
      }
  }
  pdl_wait();                                                // X (and Y, R) are written by earlier kernels
  {
    const float* X = a.X + int64_t(t) * a.xs + int64_t(a.in0) * a.n;
    for (int q = threadIdx.x; q < nin * TS; q += kSGRThreads) {
      const int c = q / TS, rr = q - c * TS, r = rr / WX, col = rr - r * WX;
      const int gx = ix0 - 1 + col, gy = iy0 - 1 + r;
      const bool ok = gx >= 0 && gx < n1 && gy >= 0 && gy < n1;
      cp_async_elem(Xs + q, ok ? X + int64_t(c) * a.n + int64_t(gy) * n1 + gx : X, ok);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  }
  pdl_trigger();
  float off[P];
#pragma unroll
  for (int b = 0; b < P; ++b) off[b] = 0.0f;
  const float* win = Xs + ty * WX + tx;                      // this node's 3 x 3 window in column in0
  const int o0 = a.out0, o1 = a.out1, kmax = a.kmax;
  static_for(std::make_integer_sequence<int, P>{}, [&](auto ia) {
    constexpr int A = decltype(ia)::value;
    if (A < a.in0 || A >= a.in1) return;
    const float* w = win + (A - a.in0) * TS;
    const float SW = w[0], S = w[1], SE = w[2];
    const float W = w[WX], C = w[WX + 1], E = w[WX + 2];
    const float NW = w[2 * WX], N = w[2 * WX + 1], NE = w[2 * WX + 2];
    const float c4 = 4.0f * C;
    const float aS = c4 - S, aN = c4 - N;
    const float t0 = fmaf(-2.0f, SW, aS - W), t1 = fmaf(-2.0f, SE, aS - E);
    const float t2 = fmaf(-2.0f, NE, aN - E), t3 = fmaf(-2.0f, NW, aN - W);
    if (own && A >= o0 && A < o1) {
      Ds[(A - o0) * kSGRThreads + threadIdx.x] = fmaf(kk[0][3], t3, fmaf(kk[0][2], t2, fmaf(kk[0][1], t1, kk[0][0] * t0)));
      if (use_m) {
        const float edges = (N + S) + (E + W), corners = (NE + NW) + (SE + SW);
        Ms[(A - o0) * kSGRThreads + threadIdx.x] = a.mass * fmaf(16.0f, C, fmaf(4.0f, edges, corners));
      }
    }
    static_for(std::make_integer_sequence<int, M>{}, [&](auto ik) {
      constexpr int K = decltype(ik)::value;               // KL index K + 1
      constexpr int UP = Tab::t.up[A][K], DN = Tab::t.dn[A][K], AK = Tab::t.idx[A][K];
      if (K + 1 >= kmax) return;
      const bool up = UP >= 0 && UP >= o0 && UP < o1;
      const bool dn = DN >= 0 && DN >= o0 && DN < o1;
      if (!up && !dn) return;
      const float u = fmaf(kk[K + 1][3], t3, fmaf(kk[K + 1][2], t2, fmaf(kk[K + 1][1], t1, kk[K + 1][0] * t0)));
      if constexpr (UP >= 0) {
        if (up) off[UP] = fmaf(a.cup[AK], u, off[UP]);
      }
      if constexpr (DN >= 0) {
        if (dn) off[DN] = fmaf(a.cup[AK - 1], u, off[DN]);
      }
    });
  });
  if (!live) return;
  const int64_t node = int64_t(iy) * n1 + ix;
  static_for(std::make_integer_sequence<int, P>{}, [&](auto ib) {
    constexpr int Bc = decltype(ib)::value;
    if (Bc < o0 || Bc >= o1) return;
    const float diag = own ? Ds[(Bc - o0) * kSGRThreads + threadIdx.x] : 0.0f;
    float out = fmaf(a.c0, diag, a.c1 * off[Bc]);
    if (use_m) out = fmaf(a.cm, Ms[(Bc - o0) * kSGRThreads + threadIdx.x], out);
    if (a.R) out = fmaf(a.cr, a.R[int64_t(t) * a.rs + int64_t(Bc - a.rcol0) * a.n + node], out);
    float* yp = a.Y + int64_t(t) * a.ys + int64_t(Bc - a.ycol0) * a.n + node;
    if (a.cy != 0.0f) out = fmaf(a.cy, *yp, out);
    *yp = out;
  });
}

// the compiled (M, p) of the register kernel: the time-dependent workload's (4, 3), where it
// is the fastest form of the full operator, and small shapes.  Not (6, 3): with one thread
// per node a 128 x 128 grid gives about three warps per SM, which cannot hide the
// instruction fetches of its fully unrolled code (ncu: 5.7 no_instruction stalls per
// issue, 37.6 us against 19.1 us for the quad kernel)
#define SGOC_SGR_SHAPES(X) X(1, 1) X(2, 2) X(3, 2) X(3, 3) X(4, 3)

static bool sgr_compiled(int M, int p) {
#define SGOC_SGR_CASE(m, q) if (M == m && p == q) return true;
  SGOC_SGR_SHAPES(SGOC_SGR_CASE)
#undef SGOC_SGR_CASE
  return false;
}

// the multi-index order the register kernel was compiled with, for a check against the
// problem's own (first `count` indices, row-major (count x M)); false when not compiled
bool sgr_indices(int M, int p, std::vector<int>& out) {
  out.clear();
#define SGOC_SGR_IDX(m, q)                                                   \
  if (M == m && p == q) {                                                    \
    constexpr const LegChaos<m, q>& c = LegTab<m, q>::t;                     \
    for (int i = 0; i < LegChaos<m, q>::P; ++i)                              \
      for (int j = 0; j < m; ++j) out.push_back(c.idx[i][j]);                \
    return true;                                                             \
  }
  SGOC_SGR_SHAPES(SGOC_SGR_IDX)
#undef SGOC_SGR_IDX
  return false;
}

template <typename T>
static bool sgr_feasible(const SGArgs<T>& a) {
  if constexpr (!std::is_same<T, float>::value) {
    return false;
  } else {
    if (a.legendre_p < 0 || !sgr_compiled(a.M, a.legendre_p)) return false;
    return sgr_smem(a.in1 - a.in0, a.out1 - a.out0, !a.no_own, a.cm != 0.0f) <= kMaxSmem;
  }
}

template <int M, int PD>
static cudaError_t launch_sgr_mp(const SGArgs<float>& a, cudaStream_t st, const SGMulti<float>& mg) {
  const size_t smem = sgr_smem(a.in1 - a.in0, a.out1 - a.out0, !a.no_own, a.cm != 0.0f);
  cudaError_t e = cudaFuncSetAttribute(sgr_kernel<M, PD>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMaxSmem));
  if (e != cudaSuccess) return e;
  dim3 grid(unsigned((a.n1 + kSGRTX - 1) / kSGRTX), unsigned((a.n1 + kSGRTY - 1) / kSGRTY),
            unsigned(a.nslabs * mg.ng));
  return launch_pdl(sgr_kernel<M, PD>, grid, dim3(kSGRThreads), smem, st, a, mg);
}

template <typename T>
static cudaError_t launch_sgr(const SGArgs<T>& a, cudaStream_t st, const SGMulti<T>& mg) {
  if constexpr (!std::is_same<T, float>::value) {
    return cudaErrorInvalidConfiguration;
  } else {
    const int nout = a.out1 - a.out0;
    const double w = 4.0, cells = double(a.n) * a.nslabs * mg.ng;
    const double bytes = w * cells * (double(a.in1 - a.in0) + nout * (1.0 + (a.R ? 1 : 0) + (a.cy != 0.0f ? 1 : 0))) +
                         w * (a.M + 1.0) * a.nx * a.nx;
    const double flops = cells * (15.0 * (a.in1 - a.in0) + 9.0 * nout + 9.0 * (a.c1 != 0.0f ? a.deg_sum : 0));
    ProfScope ps(KK_SG, st, bytes, flops);
    cudaError_t e = cudaErrorInvalidConfiguration;
#define SGOC_SGR_LAUNCH(m, q) \
    if (a.M == m && a.legendre_p == q) e = launch_sgr_mp<m, q>(a, st, mg);
    SGOC_SGR_SHAPES(SGOC_SGR_LAUNCH)
#undef SGOC_SGR_LAUNCH
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
  }
}

// ---------------------------------------------------------------------------
// SG kernel variants and the tuning cache.  All variants form the same products
// and sums in the same order, so the choice changes timing only.
//   0: one-phase kernel (tile by the heuristic), 1: quad kernel, 32-node tile,
//   2: quad kernel, 16-node tile, 3: two-phase kernel (float32, slot table),
//   4, 5: quad kernel on 32- and 16-node tiles compiled for four CTAs per SM
//   (64 registers) instead of two, 6: direct kernel (few outputs and couplings).
// The cache maps a launch shape (grid, column ranges, KL terms, truncation,
// slabs, element size, epilogue terms) to the variant measured fastest.
// ---------------------------------------------------------------------------
namespace {
struct SGKey {
  int n1, in0, in1, out0, out1, M, kmax, nslabs, esize, flags;
  bool operator<(const SGKey& o) const {
    const int a[10] = {n1, in0, in1, out0, out1, M, kmax, nslabs, esize, flags};
    const int b[10] = {o.n1, o.in0, o.in1, o.out0, o.out1, o.M, o.kmax, o.nslabs, o.esize, o.flags};
    for (int i = 0; i < 10; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};
std::mutex g_tune_mu;
std::map<SGKey, int> g_tune;

template <typename T>
SGKey sg_key(const SGArgs<T>& a) {
  const int flags = (a.cm != T(0) ? 1 : 0) | (a.R ? 2 : 0) | (a.cy != T(0) ? 4 : 0) | (a.no_own ? 8 : 0);
  return SGKey{a.n1, a.in0, a.in1, a.out0, a.out1, a.M, a.kmax, a.nslabs, int(sizeof(T)), flags};
}
}  // namespace

template <typename T>
int sg_tuned_variant(const SGArgs<T>& a) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  const auto it = g_tune.find(sg_key(a));
  return it == g_tune.end() ? -1 : it->second;
}

template <typename T>
void sg_set_variant(const SGArgs<T>& a, int v) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[sg_key(a)] = v;
}

template <typename T>
void sg_clear_variant(const SGArgs<T>& a) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune.erase(sg_key(a));
}

void sg_clear_tuning() {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune.clear();
}

template <typename T>
static bool sg_one_phase_fits(const SGArgs<T>& a) {
  return (sg_smem<T, 32>(a) <= kMaxSmem && a.n1 >= 24) || (sg_smem<T, 16>(a) <= kMaxSmem && a.n1 >= 12) ||
         sg_smem<T, 8>(a) <= kMaxSmem;
}

template <typename T>
bool sg_variant_feasible(const SGArgs<T>& a, int v) {
  switch (v) {
    case 0: return sg_one_phase_fits(a);
    case 1: case 4: return a.n1 >= 24 && a.M + 1 <= 17 && sg4_smem<T, 32>(a) <= kMaxSmem;
    case 2: case 5: return a.n1 >= 15 && a.M + 1 <= 17 && sg4_smem<T, 16>(a) <= kMaxSmem;
    case 3:
      if constexpr (std::is_same<T, float>::value)
        return a.u_mb && a.n1 >= 24 && a.M + 1 <= 17 && sgu_smem(a) + 4096 <= kMaxSmem;
      return false;
    case 6:                                   // its work grows with outputs x (1 + couplings); it is
                                              // also the only form when no staged form fits
      return double(a.out1 - a.out0) + (a.c1 != T(0) ? a.deg_sum : 0.0) <= kSGDirectMaxTerms ||
             !sg_one_phase_fits(a);
    case 7: return sgr_feasible(a);
    default: return false;
  }
}

template <typename T>
static cudaError_t launch_sg_one_phase(const SGArgs<T>& a, cudaStream_t st, const SGMulti<T>& mg) {
  size_t s32 = sg_smem<T, 32>(a), s16 = sg_smem<T, 16>(a), s8 = sg_smem<T, 8>(a);
  if (s32 <= kMaxSmem && a.n1 >= 24) return launch_sg_tx<T, 32>(a, s32, st, mg);
  if (s16 <= kMaxSmem && a.n1 >= 12) return launch_sg_tx<T, 16>(a, s16, st, mg);
  if (s8 <= kMaxSmem) return launch_sg_tx<T, 8>(a, s8, st, mg);
  return cudaErrorInvalidConfiguration;
}

template <typename T>
cudaError_t launch_sg_variant(const SGArgs<T>& a, int v, cudaStream_t st, const SGMulti<T>* mgp) {
  if (a.out1 <= a.out0 || a.nslabs <= 0) return cudaSuccess;
  if (!a.no_own && (a.out0 < a.in0 || a.out1 > a.in1)) return cudaErrorInvalidValue;
  if (!sg_variant_feasible(a, v)) return cudaErrorInvalidConfiguration;
  const SGMulti<T>& mg = mgp ? *mgp : sg_solo<T>();
  switch (v) {
    case 1: return launch_sg4_tx<T, 32, 2>(a, sg4_smem<T, 32>(a), st, mg);
    case 2: return launch_sg4_tx<T, 16, 2>(a, sg4_smem<T, 16>(a), st, mg);
    case 4: return launch_sg4_tx<T, 32, 4>(a, sg4_smem<T, 32>(a), st, mg);
    case 5: return launch_sg4_tx<T, 16, 4>(a, sg4_smem<T, 16>(a), st, mg);
    case 6: return launch_sgd<T>(a, st, mg);
    case 7: return launch_sgr<T>(a, st, mg);
    case 3:
      if constexpr (std::is_same<T, float>::value) {
        cudaError_t e = cudaSuccess;
        if (try_launch_sgu(a, st, &e, mg)) return e;
      }
      return cudaErrorInvalidConfiguration;
    default: return launch_sg_one_phase<T>(a, st, mg);
  }
}

// the kernel for a launch shape: the tuned variant, else the built-in rule
template <typename T>
static int sg_choose(const SGArgs<T>& a) {
  const int tuned = sg_tuned_variant(a);
  if (tuned >= 0 && sg_variant_feasible(a, tuned)) return tuned;
  // untuned: the quad kernel on 32-node tiles (measured fastest at 128x128 P=84 and 512x512
  // P=165 in float32), on 16-node tiles for narrower grids, else one-phase
  if (sg_variant_feasible(a, 1)) return 1;
  if (sg_variant_feasible(a, 2)) return 2;
  if (sg_one_phase_fits(a)) return 0;
  // no staged form fits shared memory (hundreds of float64 input columns, e.g. P = 495):
  // the direct form needs none and applies to every shape
  return 6;
}

template <typename T>
cudaError_t launch_sg(const SGArgs<T>& a, cudaStream_t st) {
  if (a.out1 <= a.out0 || a.nslabs <= 0) return cudaSuccess;
  if (!a.no_own && (a.out0 < a.in0 || a.out1 > a.in1)) return cudaErrorInvalidValue;
  return launch_sg_variant(a, sg_choose(a), st);
}

template <typename T>
cudaError_t launch_sg_group(const SGArgs<T>* a, int ng, cudaStream_t st) {
  if (ng == 1) return launch_sg(a[0], st);
  if (ng < 1 || ng > kMaxGroup) return cudaErrorInvalidValue;
  if (a[0].out1 <= a[0].out0 || a[0].nslabs <= 0) return cudaSuccess;
  if (!a[0].no_own && (a[0].out0 < a[0].in0 || a[0].out1 > a[0].in1)) return cudaErrorInvalidValue;
  SGMulti<T> mg{};
  mg.ng = ng;
  for (int g = 0; g < ng; ++g) {
    mg.X[g] = a[g].X; mg.Y[g] = a[g].Y; mg.R[g] = a[g].R; mg.kap[g] = a[g].kap;
    mg.c0[g] = a[g].c0; mg.c1[g] = a[g].c1; mg.cm[g] = a[g].cm; mg.cr[g] = a[g].cr;
  }
  return launch_sg_variant(a[0], sg_choose(a[0]), st, &mg);
}

// ---------------------------------------------------------------------------
// Mass-matrix combinations (Eq. (def-Mcal): M_cal = I (x) M, M_gamma = H^gamma (x) M)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T mass_apply(const T* __restrict__ V, int ix, int iy, int n1, T mass) {
  const T C = V[iy * n1 + ix];
  const T N = ldz(V, ix, iy + 1, n1), S = ldz(V, ix, iy - 1, n1);
  const T E = ldz(V, ix + 1, iy, n1), Wv = ldz(V, ix - 1, iy, n1);
  const T NE = ldz(V, ix + 1, iy + 1, n1), NW = ldz(V, ix - 1, iy + 1, n1);
  const T SE = ldz(V, ix + 1, iy - 1, n1), SW = ldz(V, ix - 1, iy - 1, n1);
  const T edges = (N + S) + (E + Wv);
  const T corners = (NE + NW) + (SE + SW);
  return mass * fma(T(16), C, fma(T(4), edges, corners));
}

// One thread owns node column ix of a strip of kMassRows rows of one chaos column
// and slab; it walks the strip keeping the centre value c(y) and the horizontal
// pair h(y) = V(x-1,y) + V(x+1,y) of three consecutive rows, so every output
// (h^2/36)(16 c(y) + 4 (c(y-1) + c(y+1) + h(y)) + h(y-1) + h(y+1)) costs three
// coalesced loads.  blockIdx.y runs over (strip, column, slab) work items.
constexpr int kMassRows = 8;

template <typename T>
__device__ __forceinline__ void mass_row(const T* __restrict__ V, int ix, int y, int n1, T& c, T& h) {
  if (y < 0 || y >= n1) { c = T(0); h = T(0); return; }
  const T* row = V + int64_t(y) * n1;
  c = row[ix];
  h = (ix > 0 ? row[ix - 1] : T(0)) + (ix + 1 < n1 ? row[ix + 1] : T(0));
}

// TX: nodes per tile row (= threads per CTA): 128, or 64 / 32 on narrower grids so that
// no thread and no staged column is idle
template <typename T, int TX>
__global__ void __launch_bounds__(TX) mass_kernel(MassArgs<T> a, int strips, int64_t nwork) {
  pdl_enter();
  // tile of the inputs: rows y0-1 .. y0+kMassRows, columns x0-1 .. x0+TX (zero outside the grid)
  constexpr int TW = TX + 2, TH = kMassRows + 2;
  __shared__ T Vs[3][TH][TW];
  const int n1 = a.n1;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX;
  const int ix = x0 + tid;
  for (int64_t w = blockIdx.y; w < nwork; w += gridDim.y) {
    const int strip = int(w % strips);
    const int64_t cq = w / strips;
    const int c = int(cq % a.ncols);
    const int t = int(cq / a.ncols);
    const int y0 = strip * kMassRows;
    const int ny = min(kMassRows, n1 - y0);
    const int col = a.col0 + c;
    const T hg = col == 0 ? T(1) : T(1) + a.gamma;
    const T dt = (a.nt > 1 && (t == 0 || t == a.nt - 1)) ? T(0.5) : T(1);
    // stage every input's tile with independent loads
    for (int j = 0; j < a.nv; ++j) {
      const int ts = t + a.shift[j];
      if (ts < 0 || ts >= a.nslabs) continue;
      const T* V = a.V[j] + int64_t(ts) * a.vs[j] + int64_t(c) * a.n;
      for (int q = tid; q < TH * TW; q += TX) {
        const int r = q / TW, xx = q - r * TW;
        const int gy = y0 - 1 + r, gx = x0 - 1 + xx;
        Vs[j][r][xx] = (gy >= 0 && gy < n1 && gx >= 0 && gx < n1) ? V[int64_t(gy) * n1 + gx] : T(0);
      }
    }
    __syncthreads();
    if (ix < n1) {
      T* op = a.out + int64_t(t) * a.os + int64_t(c) * a.n + int64_t(y0) * n1 + ix;
      T acc[kMassRows];
#pragma unroll
      for (int r = 0; r < kMassRows; ++r) acc[r] = (r < ny && a.cy != T(0)) ? a.cy * op[int64_t(r) * n1] : T(0);
      for (int j = 0; j < a.nv; ++j) {
        const int ts = t + a.shift[j];
        if (ts < 0 || ts >= a.nslabs) continue;
        T wj = a.a[j];
        if (a.wflags[j] & 1) wj *= hg;
        if (a.wflags[j] & 2) wj *= dt;
        wj *= a.mass;
        const T(*tile)[TW] = Vs[j];
        const int xx = tid + 1;
        T cm = tile[0][xx], hm = tile[0][xx - 1] + tile[0][xx + 1];
        T c0 = tile[1][xx], h0 = tile[1][xx - 1] + tile[1][xx + 1];
#pragma unroll
        for (int r = 0; r < kMassRows; ++r) {
          const T cp = tile[r + 2][xx], hp = tile[r + 2][xx - 1] + tile[r + 2][xx + 1];
          const T edges = (cm + cp) + h0;
          const T corners = hm + hp;
          acc[r] = fma(wj, fma(T(16), c0, fma(T(4), edges, corners)), acc[r]);
          cm = c0; hm = h0; c0 = cp; h0 = hp;
        }
      }
      if (a.R) {
        const T* Rp = a.R + int64_t(t) * a.rs + int64_t(c) * a.n + int64_t(y0) * n1 + ix;
#pragma unroll
        for (int r = 0; r < kMassRows; ++r)
          if (r < ny) acc[r] = fma(a.ar, Rp[int64_t(r) * n1], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < kMassRows; ++r)
        if (r < ny) op[int64_t(r) * n1] = acc[r];
    }
    __syncthreads();                                  // the tile is rewritten by the next work item
  }
}

static int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  const int64_t cap = 152 * 32;
  return int(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
cudaError_t launch_mass(const MassArgs<T>& a, cudaStream_t st) {
  const int64_t total = int64_t(a.nslabs) * a.ncols * a.n;
  if (total == 0) return cudaSuccess;
  const double w = sizeof(T);
  ProfScope ps(KK_MASS, st, w * total * (a.nv + 1 + (a.cy != T(0) ? 1 : 0) + (a.R ? 1 : 0)),
               double(total) * (20.0 * a.nv + 2.0));
  // one tile of tx nodes per CTA and strip: the narrowest of 128 / 64 / 32 that spans a row
  // (or 128 on wider grids)
  const int tx = a.n1 <= 32 ? 32 : a.n1 <= 64 ? 64 : 128;
  const int strips = (a.n1 + kMassRows - 1) / kMassRows;
  const int64_t nwork = int64_t(strips) * a.ncols * a.nslabs;
  const dim3 grid(unsigned((a.n1 + tx - 1) / tx), unsigned(nwork < 65535 ? nwork : 65535));
  {
    const cudaError_t le_ =
        tx == 32 ? launch_pdl(mass_kernel<T, 32>, dim3(grid), dim3(tx), size_t(0), st, a, strips, nwork)
        : tx == 64 ? launch_pdl(mass_kernel<T, 64>, dim3(grid), dim3(tx), size_t(0), st, a, strips, nwork)
                   : launch_pdl(mass_kernel<T, 128>, dim3(grid), dim3(tx), size_t(0), st, a, strips, nwork);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Chebyshev semi-iteration for the mass blocks (Sec. 2, Sec. 5: Chebyshev-5)
// x_{k+1} = omega_{k+1} (D^{-1}(b - M x_k) + x_k - x_{k-1}) + x_{k-1},
// omega_1 = 1, omega_2 = 2/(2 - rho^2), omega_{k+1} = 1/(1 - rho^2 omega_k / 4).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T cheb_scale(const ChebArgs<T>& a, int64_t col) {
  if (a.scale_mode == 2) return a.scale;
  if (a.scale_mode != 1) return T(1);
  const int64_t sp = int64_t(a.slabs) * a.P;
  const int64_t blk = col / sp, cc = col % sp;
  const int t = int(cc / a.P), al = int(cc % a.P);
  T s = a.nt > 0 ? a.tau * ((a.nt > 1 && (t == 0 || t == a.nt - 1)) ? T(0.5) : T(1)) : T(1);
  s *= blk == 0 ? (al == 0 ? T(1) : T(1) + a.gamma) : a.beta;
  return T(1) / s;
}

// ---------------------------------------------------------------------------
// Exact mass solve.  M = M1 (x) M1 (x fastest), M1 = L D L^T with L unit lower bidiagonal
// (subdiagonal l_i) and D diagonal (reciprocals id_i): solve along y (a thread per grid
// column x, coalesced across the warp), then along x (a CTA stages kMassRows rows of a
// column in shared memory, a thread solves one row there), with the block scaling.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) mass_exact_y_kernel(const T* __restrict__ B, T* X, int n1, int64_t n,
                                                          const T* __restrict__ l, const T* __restrict__ id) {
  pdl_enter();
  const int ix = blockIdx.x * 128 + threadIdx.x;
  if (ix >= n1) return;
  const T* b = B + int64_t(blockIdx.y) * n + ix;
  T* x = X + int64_t(blockIdx.y) * n + ix;
  T z = b[0];
  x[0] = z;
  for (int iy = 1; iy < n1; ++iy) {                    // L z = b
    z = fma(-l[iy], z, b[int64_t(iy) * n1]);
    x[int64_t(iy) * n1] = z;
  }
  T v = z * id[n1 - 1];                                 // L^T x = D^{-1} z
  x[int64_t(n1 - 1) * n1] = v;
  for (int iy = n1 - 2; iy >= 0; --iy) {
    v = fma(-l[iy + 1], v, x[int64_t(iy) * n1] * id[iy]);
    x[int64_t(iy) * n1] = v;
  }
}

template <typename T>
__global__ void mass_exact_x_kernel(ChebArgs<T> a, const T* __restrict__ l, const T* __restrict__ id, int rows) {
  extern __shared__ __align__(16) unsigned char mx_smem_raw[];
  T* tile = reinterpret_cast<T*>(mx_smem_raw);        // [rows][s], s odd: the rows' threads hit distinct banks
  pdl_enter();
  const int n1 = a.n1, s = n1 | 1;
  const int64_t c = blockIdx.y;
  const int y0 = blockIdx.x * rows;
  const int nr = min(rows, n1 - y0);
  T* X = a.X + c * a.n + int64_t(y0) * n1;
  for (int q = threadIdx.x; q < nr * n1; q += blockDim.x) {
    const int r = q / n1, x = q - r * n1;
    tile[r * s + x] = X[q];
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    T* row = tile + threadIdx.x * s;
    T z = row[0];
    for (int ix = 1; ix < n1; ++ix) { z = fma(-l[ix], z, row[ix]); row[ix] = z; }
    T v = z * id[n1 - 1];
    row[n1 - 1] = v;
    for (int ix = n1 - 2; ix >= 0; --ix) { v = fma(-l[ix + 1], v, row[ix] * id[ix]); row[ix] = v; }
  }
  __syncthreads();
  const T sc = cheb_scale(a, c);
  for (int q = threadIdx.x; q < nr * n1; q += blockDim.x) {
    const int r = q / n1, x = q - r * n1;
    X[q] = sc * tile[r * s + x];
  }
}

template <typename T>
cudaError_t launch_mass_exact(const ChebArgs<T>& a, const T* l, const T* id, cudaStream_t st) {
  if (a.ncols == 0) return cudaSuccess;
  if (a.ncols > 65535) return cudaErrorInvalidValue;
  ProfScope ps(KK_CHEB, st, double(sizeof(T)) * a.n * a.ncols * 4, double(a.n) * a.ncols * 8);
  cudaError_t e = launch_pdl(mass_exact_y_kernel<T>, dim3(unsigned((a.n1 + 127) / 128), unsigned(a.ncols)), dim3(128),
                             size_t(0), st, a.B, a.X, a.n1, a.n, l, id);
  if (e != cudaSuccess) return e;
  note_launch();
  const int s = a.n1 | 1;
  int rows = int(std::max<int64_t>(1, std::min<int64_t>(32, (48 * 1024) / (int64_t(s) * sizeof(T)))));
  const int threads = std::max(32, ((rows + 31) / 32) * 32);
  e = launch_pdl(mass_exact_x_kernel<T>, dim3(unsigned((a.n1 + rows - 1) / rows), unsigned(a.ncols)), dim3(threads),
                 size_t(rows) * s * sizeof(T), st, a, l, id, rows);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// omega_{k+1} of the Golub-Varga recurrence (omega_1 = 1), in float64 on host and device alike
__host__ __device__ __forceinline__ double cheb_omega(int k, double rho, double prev) {
  if (k == 0) return 1.0;
  if (k == 1) return 2.0 / (2.0 - rho * rho);
  return 1.0 / (1.0 - rho * rho * prev / 4.0);
}

struct ChebWeights { float om[64]; };   // omega_{k+1}, k < steps <= 64, from the host

// float32, all steps for one column in one CTA: x_k lives in shared memory with a
// zero border (pitch n1 + 2).  Thread (tx, ty) owns the vertical strip of NPT
// consecutive rows ty*NPT .. of column tx and keeps x_{k-1} and x_{k+1} of its
// nodes in registers; it walks the strip with a three-row window (x-1, x, x+1
// of rows y-1, y, y+1), so each stencil costs three shared-memory loads.  Same
// arithmetic (and summation order) as the per-step kernel below.
template <int NPT>
__global__ void __launch_bounds__(1024, 1) cheb_fused_kernel(ChebArgs<float> a, float dinv, ChebWeights w) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char cheb_smem[];
  float* S = reinterpret_cast<float*>(cheb_smem);
  const int n1 = a.n1, pitch = n1 + 2;
  const int n = n1 * n1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * blockDim.x + tx, nt = blockDim.x * blockDim.y;
  const int y0 = ty * NPT;
  const int ny = tx < n1 ? max(0, min(NPT, n1 - y0)) : 0;     // rows of this thread
  const float mass = a.mass;
  // the zero border: rows 0 and n1+1, columns 0 and n1+1 (interiors are written before they are read)
  for (int q = tid; q < 4 * (n1 + 1); q += nt) {
    const int side = q / (n1 + 1), pos = q - side * (n1 + 1);
    const int o = side == 0 ? pos : side == 1 ? (n1 + 1) * pitch + pos + 1 : side == 2 ? (pos + 1) * pitch : pos * pitch + n1 + 1;
    S[o] = 0.f;
  }
  for (int64_t col = blockIdx.x; col < a.ncols; col += gridDim.x) {
    const float* __restrict__ B = a.B + col * n + int64_t(y0) * n1 + tx;
    float* __restrict__ O = a.X + col * n + int64_t(y0) * n1 + tx;
    const float sc = cheb_scale(a, col);
    float xp[NPT], xn[NPT];
    // x_1 = D^{-1} b (x_0 = 0)
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      xp[j] = 0.f;
      xn[j] = j < ny ? dinv * B[j * n1] : 0.f;
    }
    if (a.steps == 1) {
      pdl_trigger();
#pragma unroll
      for (int j = 0; j < NPT; ++j)
        if (j < ny) O[j * n1] = sc * xn[j];
    } else {
      __syncthreads();                                   // the previous column's last reads are done
#pragma unroll
      for (int j = 0; j < NPT; ++j)
        if (j < ny) S[(y0 + j + 1) * pitch + tx + 1] = xn[j];
    }
    for (int k = 1; k < a.steps; ++k) {
      __syncthreads();
      const bool last = k == a.steps - 1;
      if (last) pdl_trigger();
      const float om = w.om[k];
      if (ny > 0) {
        const float* p = S + y0 * pitch + tx;            // row y0 - 1 (padded row y0), column x - 1
        float l0 = p[0], c0 = p[1], r0 = p[2];
        p += pitch;
        float l1 = p[0], c1 = p[1], r1 = p[2];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
          if (j < ny) {
            p += pitch;
            const float l2 = p[0], c2 = p[1], r2 = p[2];
            const float edges = (c2 + c0) + (r1 + l1);
            const float corners = (r2 + l2) + (r0 + l0);
            const float r = B[j * n1] - mass * fmaf(16.f, c1, fmaf(4.f, edges, corners));
            xn[j] = fmaf(om, fmaf(dinv, r, c1 - xp[j]), xp[j]);
            xp[j] = c1;
            l0 = l1; c0 = c1; r0 = r1;
            l1 = l2; c1 = c2; r1 = r2;
          }
        }
      }
      if (last) {
#pragma unroll
        for (int j = 0; j < NPT; ++j)
          if (j < ny) O[j * n1] = sc * xn[j];
      } else {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NPT; ++j)
          if (j < ny) S[(y0 + j + 1) * pitch + tx + 1] = xn[j];
      }
    }
  }
}

// One step for columns that do not fit in shared memory (and for float64): a
// thread walks a strip of kChebRows rows of one column with a three-row window of
// x_k (three loads per node, as in mass_kernel); blockIdx.y runs over (strip,
// column) work items.  Same arithmetic and order as mass_apply.
constexpr int kChebRows = 8;

template <typename T>
__device__ __forceinline__ void cheb_row(const T* __restrict__ X, int ix, int y, int n1, T& l, T& c, T& r) {
  if (y < 0 || y >= n1) { l = c = r = T(0); return; }
  const T* row = X + int64_t(y) * n1;
  c = row[ix];
  l = ix > 0 ? row[ix - 1] : T(0);
  r = ix + 1 < n1 ? row[ix + 1] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(128) cheb_kernel(ChebArgs<T> a, const T* __restrict__ xk, T* xkm1, T* out, T dinv,
                                                   T omega, int mode, int strips, int64_t nwork) {
  pdl_enter();
  const int n1 = a.n1;
  const int64_t n = int64_t(n1) * n1;
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= n1) return;
  for (int64_t w = blockIdx.y; w < nwork; w += gridDim.y) {
    const int strip = int(w % strips);
    const int64_t col = w / strips;
    const int y0 = strip * kChebRows;
    const int ny = min(kChebRows, n1 - y0);
    const int64_t cb = col * n;
    const T* Bc = a.B + cb;
    const T* Xc = xk + cb;
    T* xpc = xkm1 + cb;
    T* dst = out ? out + cb : xpc;
    const T sc = out ? cheb_scale(a, col) : T(1);
    if (mode == 0) {                                // x_1 = D^{-1} b (x_0 = 0)
      for (int r = 0; r < ny; ++r) {
        const int64_t node = int64_t(y0 + r) * n1 + ix;
        dst[node] = sc * (dinv * Bc[node]);
      }
      continue;
    }
    T lm, cm, rm, l0, c0, r0;
    cheb_row(Xc, ix, y0 - 1, n1, lm, cm, rm);
    cheb_row(Xc, ix, y0, n1, l0, c0, r0);
#pragma unroll
    for (int r = 0; r < kChebRows; ++r) {
      if (r >= ny) break;
      T lp, cp, rp;
      cheb_row(Xc, ix, y0 + r + 1, n1, lp, cp, rp);
      const int64_t node = int64_t(y0 + r) * n1 + ix;
      const T edges = (cp + cm) + (r0 + l0);
      const T corners = (rp + lp) + (rm + lm);
      const T res = Bc[node] - a.mass * fma(T(16), c0, fma(T(4), edges, corners));
      const T xprev = mode == 1 ? T(0) : xpc[node];
      const T x = fma(omega, fma(dinv, res, c0 - xprev), xprev);
      dst[node] = sc * x;
      lm = l0; cm = c0; rm = r0;
      l0 = lp; c0 = cp; r0 = rp;
    }
  }
}

template <typename T>
cudaError_t launch_cheb(const ChebArgs<T>& a, cudaStream_t st) {
  const int64_t total = a.ncols * a.n;
  if (total == 0) return cudaSuccess;
  const double lmin = 0.25, lmax = 2.25;
  const double gam = 0.5 * (lmin + lmax), rho = (lmax - lmin) / (lmax + lmin);
  const T dinv = T(1.0 / (gam * 16.0 * double(a.mass)));
  if constexpr (std::is_same<T, float>::value) if (a.n1 <= 127) {
    // float32 columns of up to 127 x 127 nodes: one fused launch
    const int tx = ((a.n1 + 31) / 32) * 32;
    const int by = 1024 / tx;
    const int npt = (a.n1 + by - 1) / by;                 // <= 16
    const size_t fsm = size_t(a.n1 + 2) * (a.n1 + 2) * sizeof(float);
    const ChebArgs<float>& af = a;
    auto go = [&](auto kern) -> cudaError_t {
      cudaError_t e = allow_max_smem(kern);
      if (e != cudaSuccess) return e;
      const int64_t g = a.ncols < 65535 ? a.ncols : 65535;
      // algorithmic: b read and x written once, the iterates stay on chip
      ProfScope ps(KK_CHEB, st, double(sizeof(T)) * total * 2.0, double(total) * (1.0 + 24.0 * (a.steps - 1)));
      ChebWeights wts{};
      double om = 1.0;
      for (int k = 0; k < a.steps && k < 64; ++k) { om = cheb_omega(k, rho, om); wts.om[k] = float(om); }
      {
        const cudaError_t le_ = launch_pdl(kern, dim3(unsigned(g)), (dim3(tx, by)), size_t(fsm), st,
                                          af, float(dinv), wts);
        if (le_ != cudaSuccess) return le_;
      }
      note_launch();
      return cudaGetLastError();
    };
    if (npt <= 1) return go(cheb_fused_kernel<1>);
    if (npt <= 4) return go(cheb_fused_kernel<4>);
    return go(cheb_fused_kernel<16>);
  }
  const int tx = a.n1 >= 128 ? 128 : ((a.n1 + 31) / 32) * 32;
  const int strips = (a.n1 + kChebRows - 1) / kChebRows;
  const int64_t nwork = int64_t(strips) * a.ncols;
  const dim3 grid(unsigned((a.n1 + tx - 1) / tx), unsigned(nwork < 65535 ? nwork : 65535));
  double omega = 1.0;
  // x_{k+1} is written over x_{k-1}: x_1 -> A, x_2 -> B, x_3 -> A, ...
  for (int k = 0; k < a.steps; ++k) {
    omega = cheb_omega(k, rho, omega);
    T* dst = (k % 2 == 0) ? a.tmpA : a.tmpB;      // buffer receiving x_{k+1}
    const T* xk = (k % 2 == 0) ? a.tmpB : a.tmpA; // x_k
    T* out = (k == a.steps - 1) ? a.X : nullptr;
    const int mode = k == 0 ? 0 : (k == 1 ? 1 : 2);
    ProfScope ps(KK_CHEB, st, double(sizeof(T)) * total * (2 + mode), double(total) * (mode == 0 ? 1.0 : 24.0));
    {
      const cudaError_t le_ = launch_pdl(cheb_kernel<T>, dim3(grid), dim3(tx), size_t(0), st,
                                        a, xk, dst, out, dinv, T(omega), mode, strips, nwork);
      if (le_ != cudaSuccess) return le_;
    }
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Geometric multigrid for the mean operator: constant 9-point stencils.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T stencil_apply(const T* __restrict__ X, int ix, int iy, int n1, T d, T e, T c) {
  const T C = X[iy * n1 + ix];
  const T edges = (ldz(X, ix, iy + 1, n1) + ldz(X, ix, iy - 1, n1)) + (ldz(X, ix + 1, iy, n1) + ldz(X, ix - 1, iy, n1));
  const T corners = (ldz(X, ix + 1, iy + 1, n1) + ldz(X, ix - 1, iy + 1, n1)) +
                    (ldz(X, ix + 1, iy - 1, n1) + ldz(X, ix - 1, iy - 1, n1));
  return fma(d, C, fma(e, edges, c * corners));
}

// Level-wise multigrid passes (levels above the fused V-cycle): a CTA stages the
// tile of x its strip of kMassRows rows of one column needs (independent loads,
// zero outside the grid) and each thread computes one grid column of the strip;
// blockIdx.y runs over (strip, column) work items.  Stencil order as stencil_apply.
template <typename T>
__device__ __forceinline__ T tile_stencil(const T (*Xs)[130], int r, int xx, T d, T e, T c) {
  const T C = Xs[r + 1][xx];
  const T edges = (Xs[r + 2][xx] + Xs[r][xx]) + (Xs[r + 1][xx + 1] + Xs[r + 1][xx - 1]);
  const T corners = (Xs[r + 2][xx + 1] + Xs[r + 2][xx - 1]) + (Xs[r][xx + 1] + Xs[r][xx - 1]);
  return fma(d, C, fma(e, edges, c * corners));
}

template <typename T>
__device__ __forceinline__ void stage_tile(T (*Xs)[130], const T* __restrict__ X, int n1, int x0, int y0) {
  constexpr int TW = 130, TH = kMassRows + 2;
  for (int q = threadIdx.x; q < TH * TW; q += 128) {
    const int r = q / TW, xx = q - r * TW;
    const int gy = y0 - 1 + r, gx = x0 - 1 + xx;
    Xs[r][xx] = (gy >= 0 && gy < n1 && gx >= 0 && gx < n1) ? X[int64_t(gy) * n1 + gx] : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) smooth_kernel(const T* __restrict__ b, const T* __restrict__ xin, T* xout,
                                                     int n1, T d, T e, T c, T omega, T* acc, int64_t acc_ss,
                                                     int acc_L, int acc_col0, int strips, int64_t nwork) {
  pdl_enter();
  __shared__ T Xs[kMassRows + 2][130];
  const int64_t n = int64_t(n1) * n1;
  const T wd = omega / d;
  const int tid = threadIdx.x, x0 = blockIdx.x * 128, ix = x0 + tid;
  for (int64_t w = blockIdx.y; w < nwork; w += gridDim.y) {
    const int strip = int(w % strips);
    const int64_t col = w / strips;
    const int y0 = strip * kMassRows, ny = min(kMassRows, n1 - y0);
    if (xin) {
      stage_tile(Xs, xin + col * n, n1, x0, y0);
      __syncthreads();
    }
    if (ix < n1) {
      const T* bc = b + col * n;
      T* dst = acc ? acc + (col / acc_L) * acc_ss + (acc_col0 + col % acc_L) * n : xout + col * n;
      for (int r = 0; r < ny; ++r) {
        const int64_t node = int64_t(y0 + r) * n1 + ix;
        const T x = xin ? fma(wd, bc[node] - tile_stencil(Xs, r, tid + 1, d, e, c), Xs[r + 1][tid + 1]) : wd * bc[node];
        if (acc) dst[node] += x;
        else dst[node] = x;
      }
    }
    if (xin) __syncthreads();                        // the tile is rewritten by the next work item
  }
}

template <typename T>
__global__ void __launch_bounds__(128) residual_kernel(const T* __restrict__ b, const T* __restrict__ x, T* r, int n1,
                                                       T d, T e, T c, int strips, int64_t nwork) {
  pdl_enter();
  __shared__ T Xs[kMassRows + 2][130];
  const int64_t n = int64_t(n1) * n1;
  const int tid = threadIdx.x, x0 = blockIdx.x * 128, ix = x0 + tid;
  for (int64_t w = blockIdx.y; w < nwork; w += gridDim.y) {
    const int strip = int(w % strips);
    const int64_t col = w / strips;
    const int y0 = strip * kMassRows, ny = min(kMassRows, n1 - y0);
    stage_tile(Xs, x + col * n, n1, x0, y0);
    __syncthreads();
    if (ix < n1)
      for (int rr = 0; rr < ny; ++rr) {
        const int64_t node = col * n + int64_t(y0 + rr) * n1 + ix;
        r[node] = b[node] - tile_stencil(Xs, rr, tid + 1, d, e, c);
      }
    __syncthreads();
  }
}

// full weighting = transpose of bilinear prolongation: coarse interior (I,J) sits on
// fine interior (2I+1, 2J+1); weights 1, 1/2, 1/4.
template <typename T>
__global__ void restrict_kernel(const T* __restrict__ r, T* bc, int64_t B, int n1f) {
  pdl_enter();
  const int n1c = (n1f - 1) / 2;
  const int64_t nf = int64_t(n1f) * n1f, nc = int64_t(n1c) * n1c;
  const int64_t total = B * nc;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t col = q / nc, node = q % nc;
    const int I = int(node % n1c), J = int(node / n1c);
    const T* R = r + col * nf;
    const int fx = 2 * I + 1, fy = 2 * J + 1;
    const T cen = R[fy * n1f + fx];
    const T edg = (R[(fy + 1) * n1f + fx] + R[(fy - 1) * n1f + fx]) + (R[fy * n1f + fx + 1] + R[fy * n1f + fx - 1]);
    const T cor = (R[(fy + 1) * n1f + fx + 1] + R[(fy + 1) * n1f + fx - 1]) +
                  (R[(fy - 1) * n1f + fx + 1] + R[(fy - 1) * n1f + fx - 1]);
    bc[q] = cen + T(0.5) * edg + T(0.25) * cor;
  }
}

// bilinear interpolation: fine interior i (grid node i+1); even grid node -> coarse node,
// odd -> mean of the two neighbouring coarse nodes (boundary values are zero).
template <typename T>
__device__ __forceinline__ T ldc(const T* X, int I, int J, int n1c) {
  return (I >= 0 && I < n1c && J >= 0 && J < n1c) ? X[J * n1c + I] : T(0);
}

template <typename T>
__global__ void prolong_kernel(const T* __restrict__ xc, T* xf, int64_t B, int n1f) {
  pdl_enter();
  const int n1c = (n1f - 1) / 2;
  const int64_t nf = int64_t(n1f) * n1f, nc = int64_t(n1c) * n1c;
  const int64_t total = B * nf;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t col = q / nf, node = q % nf;
    const int i = int(node % n1f), j = int(node / n1f);
    const T* X = xc + col * nc;
    const int gi = i + 1, gj = j + 1;     // fine grid node
    T v;
    if ((gi & 1) == 0 && (gj & 1) == 0) {
      v = X[(gj / 2 - 1) * n1c + gi / 2 - 1];
    } else if ((gi & 1) == 0) {
      v = T(0.5) * (ldc(X, gi / 2 - 1, (gj - 1) / 2 - 1, n1c) + ldc(X, gi / 2 - 1, (gj + 1) / 2 - 1, n1c));
    } else if ((gj & 1) == 0) {
      v = T(0.5) * (ldc(X, (gi - 1) / 2 - 1, gj / 2 - 1, n1c) + ldc(X, (gi + 1) / 2 - 1, gj / 2 - 1, n1c));
    } else {
      v = T(0.25) * ((ldc(X, (gi - 1) / 2 - 1, (gj - 1) / 2 - 1, n1c) + ldc(X, (gi + 1) / 2 - 1, (gj - 1) / 2 - 1, n1c)) +
                     (ldc(X, (gi - 1) / 2 - 1, (gj + 1) / 2 - 1, n1c) + ldc(X, (gi + 1) / 2 - 1, (gj + 1) / 2 - 1, n1c)));
    }
    xf[q] += v;
  }
}

template <typename T>
__global__ void scale_kernel(const T* __restrict__ b, T* x, int64_t cnt, T a) {
  pdl_enter();
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < cnt; q += int64_t(gridDim.x) * blockDim.x)
    x[q] = a * b[q];
}

template <typename T>
cudaError_t launch_smooth(const T* b, const T* xin, T* xout, int64_t B, int n1, Stencil s, T omega, T* acc,
                          int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st) {
  const int64_t total = B * int64_t(n1) * n1;
  if (total == 0) return cudaSuccess;
  ProfScope ps(KK_SMOOTH, st, double(sizeof(T)) * total * (xin ? 3 : 2) + (acc ? double(sizeof(T)) * total : 0.0),
               double(total) * (xin ? 21.0 : 1.0));
  const int strips = (n1 + kMassRows - 1) / kMassRows;
  const int64_t nwork = int64_t(strips) * B;
  {
    const cudaError_t le_ = launch_pdl(smooth_kernel<T>, dim3(unsigned((n1 + 127) / 128), unsigned(nwork < 65535 ? nwork : 65535)),
                                      dim3(128), size_t(0), st, b, xin, xout, n1, T(s.diag), T(s.edge), T(s.corner),
                                      omega, acc, acc_ss, acc_L, acc_col0, strips, nwork);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const T* b, const T* x, T* r, int64_t B, int n1, Stencil s, cudaStream_t st) {
  const int64_t total = B * int64_t(n1) * n1;
  if (total == 0) return cudaSuccess;
  ProfScope ps(KK_RESIDUAL, st, double(sizeof(T)) * total * 3, double(total) * 18.0);
  const int strips = (n1 + kMassRows - 1) / kMassRows;
  const int64_t nwork = int64_t(strips) * B;
  {
    const cudaError_t le_ = launch_pdl(residual_kernel<T>, dim3(unsigned((n1 + 127) / 128), unsigned(nwork < 65535 ? nwork : 65535)),
                                      dim3(128), size_t(0), st, b, x, r, n1, T(s.diag), T(s.edge), T(s.corner),
                                      strips, nwork);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const T* r, T* bc, int64_t B, int n1f, cudaStream_t st) {
  const int n1c = (n1f - 1) / 2;
  const int64_t total = B * int64_t(n1c) * n1c;
  if (total == 0) return cudaSuccess;
  ProfScope ps(KK_RESTRICT, st, double(sizeof(T)) * total * 5, double(total) * 12.0);
  {
    const cudaError_t le_ = launch_pdl(restrict_kernel<T>, dim3(grid_for(total, 256)), dim3(256), size_t(0), st,
                                      r, bc, B, n1f);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const T* xc, T* xf, int64_t B, int n1f, cudaStream_t st) {
  const int64_t total = B * int64_t(n1f) * n1f;
  if (total == 0) return cudaSuccess;
  ProfScope ps(KK_PROLONG, st, double(sizeof(T)) * total * 2.25, double(total) * 3.0);
  {
    const cudaError_t le_ = launch_pdl(prolong_kernel<T>, dim3(grid_for(total, 256)), dim3(256), size_t(0), st,
                                      xc, xf, B, n1f);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(const T* b, T* x, int64_t cnt, T a, cudaStream_t st) {
  if (cnt == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, 2.0 * sizeof(T) * cnt, 0.0);
  {
    const cudaError_t le_ = launch_pdl(scale_kernel<T>, dim3(grid_for(cnt, 256)), dim3(256), size_t(0), st,
                                      b, x, cnt, a);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Full-hierarchy V-cycle, one CTA (1024 threads) per column, all levels in
// shared memory.  Every level array carries a one-node zero border (stride
// n1 + 2) so that stencil loads need no bounds checks.  Level 0 holds two
// iterate buffers (ping-pong; the idle one takes the residual), levels >= 1
// hold two iterate buffers and the right-hand side.  The level-0 right-hand
// side stays in registers: each thread owns a vertical strip of up to
// kStripRows nodes of one grid column and slides a 3x3 window down it.
// Coarse levels are processed point-parallel on a 32 x 32 thread grid.
// ---------------------------------------------------------------------------
constexpr int kVFThreads = 1024;
constexpr int kStripRows = 16;

__device__ __forceinline__ int vf_padded(int n1) { return (n1 + 2) * (n1 + 2); }


struct Strip {
  int x, y0, y1;   // column and interior rows [y0, y1) of this thread; x < 0: idle
};

__device__ __forceinline__ Strip strip_of(int n1) {
  Strip g;
  const int nchunks = (n1 + kStripRows - 1) / kStripRows;
  const int rows = (n1 + nchunks - 1) / nchunks;
  const int t = threadIdx.x;
  const int chunk = t / n1;
  g.x = (chunk < nchunks) ? t - chunk * n1 : -1;
  g.y0 = chunk * rows;
  g.y1 = min(n1, g.y0 + rows);
  return g;
}

template <typename T>
struct VFLevel { int off, n1, grp; T d, e, c, wd; };

// ---------------------------------------------------------------------------
// One-CTA-per-column V-cycle with the grid size as a template parameter: every
// level's size, stride and shared-memory offset is a compile-time constant, and
// the levels are visited by compile-time recursion.  Level l of a hierarchy with
// N1 interior nodes per side has n1(l) = (N1 + 1) / 2^l - 1 nodes per side;
// arrays carry a zero border (stride n1 + 2).  Level 0 holds two iterate buffers
// (the idle one takes the residual) and keeps its right-hand side in registers
// (16-row strips); coarse levels hold two iterates and the right-hand side, run
// point-parallel on nested thread groups (1024 / 256 / 32 threads), and fold the
// two pre-smoothing sweeps from a zero start into one pass:
// x2 = (omega/d) (2 b - (omega/d) A b).
// ---------------------------------------------------------------------------
template <int N1>
struct VT {
  static constexpr int n1(int l) { return ((N1 + 1) >> l) - 1; }
  static constexpr int s(int l) { return n1(l) + 2; }
  static constexpr int np(int l) { return s(l) * s(l); }
  static constexpr int off(int l) { return l == 0 ? 0 : off(l - 1) + np(l - 1) * (l - 1 > 0 ? 3 : 2); }
  static constexpr int nlev() { return N1 == 1 ? 1 : 1 + VT<(N1 - 1) / 2>::nlev(); }
  static constexpr int total() { return off(nlev()); }
  // threads of the border zeroing: one per position along a side, for every array
  static constexpr int border_threads(int l = 0) { return l == nlev() ? 0 : s(l) * (l > 0 ? 3 : 2) + border_threads(l + 1); }
  // threads per CTA: 1024 for a 127 x 127 top level, 256 below (four columns per SM)
  static constexpr int nb() { return N1 >= 127 ? kVFThreads : 256; }
  static constexpr int grp0(int l) { return n1(l) >= 63 ? kVFThreads : (n1(l) >= 15 ? 256 : 32); }
  static constexpr int grp(int l) { return grp0(l) < nb() ? grp0(l) : nb(); }
};
template <>
struct VT<0> {
  static constexpr int nlev() { return 0; }
};

template <int NT>
__device__ __forceinline__ void vt_sync() {
  if (NT == kVFThreads) __syncthreads();
  else if (NT > 32) asm volatile("bar.sync 1, %0;\n" ::"r"(NT) : "memory");
  else __syncwarp();
}

// coarse-level pass: 0 jacobi, 1 double sweep from zero, 2 residual
template <typename T, int N, int NT, int MODE>
__device__ __forceinline__ void vt_pass(const T* __restrict__ xs, T* __restrict__ xd, const T* __restrict__ b,
                                       T d, T e, T c, T wd) {
  constexpr int S = N + 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int y0 = 0; y0 < N; y0 += NT / 32) {
    const int y = y0 + ty;
    if (y < N) {
#pragma unroll
      for (int x0 = 0; x0 < N; x0 += 32) {
        const int x = x0 + tx;
        if (x < N) {
          const int o = (y + 1) * S + x + 1;
          const T* v = MODE == 1 ? b : xs;
          const T edges = (v[o - S] + v[o + S]) + (v[o - 1] + v[o + 1]);
          const T corners = (v[o - S - 1] + v[o - S + 1]) + (v[o + S - 1] + v[o + S + 1]);
          const T av = fma(d, v[o], fma(e, edges, c * corners));
          if (MODE == 1) xd[o] = wd * fma(T(2), b[o], -wd * av);
          else if (MODE == 2) xd[o] = b[o] - av;
          else xd[o] = fma(wd, b[o] - av, xs[o]);
        }
      }
    }
  }
}

template <typename T, int N, int NT>
__device__ __forceinline__ void vt_restrict(const T* __restrict__ R, T* __restrict__ bc) {
  constexpr int S = N + 2, NC = (N - 1) / 2, SC = NC + 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int J0 = 0; J0 < NC; J0 += NT / 32) {
    const int J = J0 + ty;
    if (J < NC) {
#pragma unroll
      for (int I0 = 0; I0 < NC; I0 += 32) {
        const int I = I0 + tx;
        if (I < NC) {
          const T* r = R + (2 * J + 2) * S + 2 * I + 2;
          const T cen = r[0];
          const T edg = (r[S] + r[-S]) + (r[1] + r[-1]);
          const T cor = (r[S + 1] + r[S - 1]) + (r[-S + 1] + r[-S - 1]);
          bc[(J + 1) * SC + I + 1] = cen + T(0.5) * edg + T(0.25) * cor;
        }
      }
    }
  }
}

template <typename T, int N, int NT>
__device__ __forceinline__ void vt_prolong(const T* __restrict__ Xc, T* __restrict__ xf) {
  constexpr int S = N + 2, NC = (N - 1) / 2, SC = NC + 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int j0 = 0; j0 < N; j0 += NT / 32) {
    const int j = j0 + ty;
    if (j < N) {
      const int gj = j + 1;
      const T* r0 = Xc + (gj >> 1) * SC;
      const T* r1 = Xc + ((gj + 1) >> 1) * SC;
#pragma unroll
      for (int i0 = 0; i0 < N; i0 += 32) {
        const int i = i0 + tx;
        if (i < N) {
          const int gi = i + 1;
          const int c0 = gi >> 1, c1 = (gi + 1) >> 1;
          xf[(j + 1) * S + i + 1] += T(0.25) * ((r0[c0] + r0[c1]) + (r1[c0] + r1[c1]));
        }
      }
    }
  }
}

// level-0 strip pass over compile-time stride S: 0 jacobi, 1 from zero, 2 residual
template <typename T, int S, int MODE>
__device__ __forceinline__ void vt_strip(const T* __restrict__ xs, T* __restrict__ xd, const T (&bv)[kStripRows],
                                        const Strip& g, T d, T e, T c, T wd) {
  if (g.x < 0) return;
  const int cr = g.y1 - g.y0;
  if (MODE == 1) {
    T* q = xd + (g.y0 + 1) * S + g.x + 1;
#pragma unroll
    for (int j = 0; j < kStripRows; ++j)
      if (j < cr) q[j * S] = wd * bv[j];
    return;
  }
  const T* p = xs + g.y0 * S + g.x;
  T wm0 = p[0], wc0 = p[1], wp0 = p[2];
  T wm1 = p[S], wc1 = p[S + 1], wp1 = p[S + 2];
  T* q = xd + (g.y0 + 1) * S + g.x + 1;
#pragma unroll
  for (int j = 0; j < kStripRows; ++j) {
    if (j < cr) {
      const T wm2 = p[(j + 2) * S], wc2 = p[(j + 2) * S + 1], wp2 = p[(j + 2) * S + 2];
      const T edges = (wc0 + wc2) + (wm1 + wp1);
      const T corners = (wm0 + wp0) + (wm2 + wp2);
      const T r = bv[j] - fma(d, wc1, fma(e, edges, c * corners));
      q[j * S] = MODE == 2 ? r : fma(wd, r, wc1);
      wm0 = wm1; wc0 = wc1; wp0 = wp1;
      wm1 = wm2; wc1 = wc2; wp1 = wp2;
    }
  }
}

// whether the V-cycle folds each level's prolongation into its first post-smoothing sweep
template <typename T>
constexpr bool kVtFuseProlong = std::is_same<T, float>::value;

// Level-0 post-smoothing sweep with two passes folded in.  PRO: every value
// read is first corrected by the prolonged coarse result xc (a quarter of the
// sum of the four nearest coarse values, exactly as vt_prolong forms it), so the
// prolongation needs no pass of its own: the corrected iterate is read only by
// the first post-smoothing sweep.  OUT: the swept values go to the global column
// gout (stored, or added when acc) instead of xd, replacing the final copy-out.
// The window's fine rows are g.y0 + w (1-based, w = 0 .. rows + 1); g.y0 is even
// (strips of kStripRows rows, or one strip from row 0), so row w reads coarse
// rows g.y0/2 + floor(w/2) and g.y0/2 + ceil(w/2).
template <typename T, int N1, bool PRO, bool OUT>
__device__ __forceinline__ void vt_strip_post(const T* __restrict__ xs, T* __restrict__ xd, const T* __restrict__ xc,
                                             T* __restrict__ gout, bool acc, const T (&bv)[kStripRows],
                                             const Strip& g, T d, T e, T c, T wd) {
  static_assert(kStripRows % 2 == 0, "strips must start on even rows");
  constexpr int S = N1 + 2, SC = (N1 - 1) / 2 + 2;
  if (g.x < 0) return;
  const int cr = g.y1 - g.y0;
  // window columns are the 1-based fine columns g.x, g.x+1, g.x+2; their coarse
  // columns lie in lo .. lo+2 (lo+2 only for odd g.x, where it is at most SC-1)
  const int lo = g.x >> 1;
  const bool odd = g.x & 1;
  const T* cp = xc + (g.y0 >> 1) * SC + lo;
  T s0[3] = {T(0), T(0), T(0)};
  // pair sums r[c0] + r[c1] of coarse row i (relative) for the three window columns
  auto csum = [&](int i, T (&s)[3]) {
    const T* q = cp + i * SC;
    const T v0 = q[0], v1 = q[1], v2 = odd ? q[2] : T(0);
    const T m0 = odd ? v1 : v0;
    s[0] = v0 + m0;
    s[1] = m0 + v1;
    s[2] = v1 + (odd ? v2 : v1);
  };
  auto wrow = [&](int w, T& m, T& cc, T& pp) {
    const T* pr = xs + (g.y0 + w) * S + g.x;
    m = pr[0]; cc = pr[1]; pp = pr[2];
    if (PRO) {
      T k[3];
      if (w & 1) {
        T s1[3];
        csum((w + 1) >> 1, s1);
#pragma unroll
        for (int q = 0; q < 3; ++q) { k[q] = T(0.25) * (s0[q] + s1[q]); s0[q] = s1[q]; }
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) k[q] = T(0.25) * (s0[q] + s0[q]);
      }
      m += k[0]; cc += k[1]; pp += k[2];
    }
  };
  T* q = xd + (g.y0 + 1) * S + g.x + 1;
  T* go = gout + g.y0 * N1 + g.x;
  // the accumulator's values are all requested before the sweep, not one latency a row
  T ga[kStripRows];
#pragma unroll
  for (int j = 0; j < kStripRows; ++j) ga[j] = (OUT && acc && j < cr) ? go[j * N1] : T(0);
  if (PRO) csum(0, s0);
  T wm0, wc0, wp0, wm1, wc1, wp1;
  wrow(0, wm0, wc0, wp0);
  wrow(1, wm1, wc1, wp1);
#pragma unroll
  for (int j = 0; j < kStripRows; ++j) {
    if (j < cr) {
      T wm2, wc2, wp2;
      wrow(j + 2, wm2, wc2, wp2);
      const T edges = (wc0 + wc2) + (wm1 + wp1);
      const T corners = (wm0 + wp0) + (wm2 + wp2);
      const T r = bv[j] - fma(d, wc1, fma(e, edges, c * corners));
      const T o = fma(wd, r, wc1);
      if (!OUT) q[j * S] = o;
      else go[j * N1] = acc ? ga[j] + o : o;
      wm0 = wm1; wc0 = wc1; wp0 = wp1;
      wm1 = wm2; wc1 = wc2; wp1 = wp2;
    }
  }
}

// ---------------------------------------------------------------------------
// The smallest levels (n1 <= 7) in one warp's registers: lane x holds grid
// column x (rows 0 .. N-1 in an array), lanes >= N hold zeros; horizontal
// neighbours come by shuffles, vertical ones from the lane's own array.  Every
// value is formed by the same operations in the same order as vt_pass,
// vt_restrict and vt_prolong (borders read as zero there and here).
// ---------------------------------------------------------------------------
constexpr unsigned kFullMask = 0xffffffffu;

// left and right neighbours of a lane's value (zero beyond the grid: lane 0 has
// no left neighbour, and lane N, the right neighbour of the last column, holds zero)
template <typename T>
__device__ __forceinline__ T wl_left(T u, int lane) {
  const T s = __shfl_up_sync(kFullMask, u, 1);
  return lane == 0 ? T(0) : s;
}
template <typename T>
__device__ __forceinline__ T wl_right(T u) { return __shfl_down_sync(kFullMask, u, 1); }

// 0 jacobi (x from xs), 1 double sweep from zero (on b), 2 residual; xd must not alias the
// array read (xs, or b for MODE 1).  The side values of rows y-1, y, y+1 slide down the column.
template <typename T, int N, int MODE>
__device__ __forceinline__ void wl_pass(const T (&xs)[N], const T (&b)[N], T (&xd)[N], int lane, T d, T e, T c,
                                        T wd) {
  const T(&v)[N] = MODE == 1 ? b : xs;
  T lm = T(0), rm = T(0);
  T l0 = wl_left(v[0], lane), r0 = wl_right(v[0]);
#pragma unroll
  for (int y = 0; y < N; ++y) {
    T l1 = T(0), r1 = T(0);
    if (y + 1 < N) { l1 = wl_left(v[y + 1], lane); r1 = wl_right(v[y + 1]); }
    const T up = y > 0 ? v[y - 1] : T(0), dn = y + 1 < N ? v[y + 1] : T(0);
    const T edges = (up + dn) + (l0 + r0);
    const T corners = (lm + rm) + (l1 + r1);
    const T av = fma(d, v[y], fma(e, edges, c * corners));
    T o;
    if (MODE == 1) o = wd * fma(T(2), b[y], -wd * av);
    else if (MODE == 2) o = b[y] - av;
    else o = fma(wd, b[y] - av, xs[y]);
    xd[y] = lane < N ? o : T(0);
    lm = l0; rm = r0; l0 = l1; r0 = r1;
  }
}

template <typename T, int N>
__device__ __forceinline__ void wl_restrict(const T (&rv)[N], T (&bc)[(N - 1) / 2], int lane) {
  constexpr int NC = (N - 1) / 2;
  T lm = wl_left(rv[0], lane), rm = wl_right(rv[0]);
#pragma unroll
  for (int J = 0; J < NC; ++J) {
    const int y = 2 * J + 1;
    const T l0 = wl_left(rv[y], lane), r0 = wl_right(rv[y]);
    const T l1 = wl_left(rv[y + 1], lane), r1 = wl_right(rv[y + 1]);
    const T cen = rv[y];
    const T edg = (rv[y + 1] + rv[y - 1]) + (r0 + l0);
    const T cor = (r1 + l1) + (rm + lm);
    const T val = cen + T(0.5) * edg + T(0.25) * cor;
    const T got = __shfl_sync(kFullMask, val, (2 * lane + 1) & 31);  // coarse column I = lane from fine 2I+1
    bc[J] = lane < NC ? got : T(0);
    lm = l1; rm = r1;
  }
}

template <typename T, int N>
__device__ __forceinline__ void wl_prolong(const T (&xc)[(N - 1) / 2], T (&xf)[N], int lane) {
  constexpr int NC = (N - 1) / 2;
  // fine column lane (1-based lane+1) reads coarse padded columns (lane+1)>>1 and (lane+2)>>1,
  // i.e. coarse lanes ((lane+1)>>1) - 1 and ((lane+2)>>1) - 1; padded column 0 is the zero border
  const int c0 = (lane + 1) >> 1, c1 = (lane + 2) >> 1;
  T A[NC], B[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const T a = __shfl_sync(kFullMask, xc[q], (c0 + 31) & 31);
    const T bq = __shfl_sync(kFullMask, xc[q], (c1 + 31) & 31);
    A[q] = c0 == 0 ? T(0) : a;
    B[q] = c1 == 0 ? T(0) : bq;                       // coarse lanes >= NC hold zeros
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const int q0 = (j + 1) >> 1, q1 = (j + 2) >> 1;   // padded coarse rows; 0 and NC+1 are borders
    const T a0 = q0 >= 1 && q0 <= NC ? A[q0 - 1] : T(0), b0 = q0 >= 1 && q0 <= NC ? B[q0 - 1] : T(0);
    const T a1 = q1 >= 1 && q1 <= NC ? A[q1 - 1] : T(0), b1 = q1 >= 1 && q1 <= NC ? B[q1 - 1] : T(0);
    const T v = xf[j] + T(0.25) * ((a0 + b0) + (a1 + b1));
    xf[j] = lane < N ? v : T(0);
  }
}

// V(nu, nu) cycle on the warp-resident levels from an N x N level down to one node
template <typename T, int N>
__device__ __forceinline__ void wl_cycle(const T (&b)[N], T (&x)[N], const VFLevel<T>* lv, int L, int nu,
                                         int lane) {
  const T d = lv[L].d, e = lv[L].e, c = lv[L].c, wd = lv[L].wd;
  if constexpr (N == 1) {
    x[0] = lane == 0 ? b[0] / d : T(0);
  } else {
    constexpr int NC = (N - 1) / 2;
    T t[N];
    if (nu == 2) {
      wl_pass<T, N, 1>(x, b, x, lane, d, e, c, wd);
    } else {
#pragma unroll
      for (int y = 0; y < N; ++y) x[y] = T(0);
      for (int sw = 0; sw < nu; ++sw) {
        wl_pass<T, N, 0>(x, b, t, lane, d, e, c, wd);
#pragma unroll
        for (int y = 0; y < N; ++y) x[y] = t[y];
      }
    }
    wl_pass<T, N, 2>(x, b, t, lane, d, e, c, wd);
    T bc[NC], xc[NC];
    wl_restrict<T, N>(t, bc, lane);
    wl_cycle<T, NC>(bc, xc, lv, L + 1, nu, lane);
    wl_prolong<T, N>(xc, x, lane);
    for (int sw = 0; sw < nu; ++sw) {
      wl_pass<T, N, 0>(x, b, t, lane, d, e, c, wd);
#pragma unroll
      for (int y = 0; y < N; ++y) x[y] = t[y];
    }
  }
}

// Coarse-level strip pass: thread t owns grid column t % N over R rows from row
// (t / N) R and slides a 3 x 3 window down it (three loads a row instead of nine
// a node).  MODE 0 jacobi, 1 double sweep from zero (window on b), 2 residual;
// PRO (MODE 0) adds the prolonged coarse result xc to every value read, as
// vt_strip_post.  The operations and their order are those of vt_pass.
template <int N, int NT>
struct CStrip {
  static constexpr int chunks = NT / N;
  static constexpr int R0 = chunks > 0 ? (N + chunks - 1) / chunks : N;
  static constexpr int R = R0 + (R0 & 1);                  // even: strips start on even rows
  static constexpr bool use = N >= 15 && chunks >= 2 && (N + R - 1) / R <= chunks;
};

template <typename T, int N, int NT, int MODE, bool PRO>
__device__ __forceinline__ void vt_cstrip(const T* __restrict__ xs, T* __restrict__ xd, const T* __restrict__ b,
                                          const T* __restrict__ xc, T d, T e, T c, T wd) {
  constexpr int R = CStrip<N, NT>::R, S = N + 2, SC = (N - 1) / 2 + 2;
  const int t = threadIdx.x;
  const int x = t % N, y0 = (t / N) * R;
  if (y0 >= N) return;
  const int ny = min(R, N - y0);
  const T* v = MODE == 1 ? b : xs;
  const int lo = x >> 1;
  const bool odd = x & 1;
  const T* cp = xc + (y0 >> 1) * SC + lo;
  T s0[3] = {T(0), T(0), T(0)};
  auto csum = [&](int i, T (&sv)[3]) {
    const T* q = cp + i * SC;
    const T v0 = q[0], v1 = q[1], v2 = odd ? q[2] : T(0);
    const T m0 = odd ? v1 : v0;
    sv[0] = v0 + m0;
    sv[1] = m0 + v1;
    sv[2] = v1 + (odd ? v2 : v1);
  };
  auto wrow = [&](int w, T& m, T& cc, T& pp) {
    const T* pr = v + (y0 + w) * S + x;
    m = pr[0]; cc = pr[1]; pp = pr[2];
    if (PRO) {
      T k[3];
      if (w & 1) {
        T s1[3];
        csum((w + 1) >> 1, s1);
#pragma unroll
        for (int q = 0; q < 3; ++q) { k[q] = T(0.25) * (s0[q] + s1[q]); s0[q] = s1[q]; }
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) k[q] = T(0.25) * (s0[q] + s0[q]);
      }
      m += k[0]; cc += k[1]; pp += k[2];
    }
  };
  if (PRO) csum(0, s0);
  T wm0, wc0, wp0, wm1, wc1, wp1;
  wrow(0, wm0, wc0, wp0);
  wrow(1, wm1, wc1, wp1);
  T* q = xd + (y0 + 1) * S + x + 1;
  const T* bq = b + (y0 + 1) * S + x + 1;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if (j < ny) {
      T wm2, wc2, wp2;
      wrow(j + 2, wm2, wc2, wp2);
      const T edges = (wc0 + wc2) + (wm1 + wp1);
      const T corners = (wm0 + wp0) + (wm2 + wp2);
      const T av = fma(d, wc1, fma(e, edges, c * corners));
      T o;
      if (MODE == 1) o = wd * fma(T(2), wc1, -wd * av);
      else if (MODE == 2) o = bq[j * S] - av;
      else o = fma(wd, bq[j * S] - av, wc1);
      q[j * S] = o;
      wm0 = wm1; wc0 = wc1; wp0 = wp1;
      wm1 = wm2; wc1 = wc2; wp1 = wp2;
    }
  }
}

// a pass of coarse level N on NT threads: the strip form where it applies
template <typename T, int N, int NT, int MODE>
__device__ __forceinline__ void vt_level_pass(const T* __restrict__ xs, T* __restrict__ xd, const T* __restrict__ b,
                                              T d, T e, T c, T wd) {
  if constexpr (CStrip<N, NT>::use) vt_cstrip<T, N, NT, MODE, false>(xs, xd, b, b, d, e, c, wd);
  else vt_pass<T, N, NT, MODE>(xs, xd, b, d, e, c, wd);
}

// One level of the cycle (coarse levels L >= 1): pre-smoothing, residual, restriction,
// the coarser levels, prolongation, post-smoothing.  Returns the buffer holding x.
template <typename T, int N1, int L, int NU>
__device__ int vt_coarse(T* base, const VFLevel<T>* lv, int nu_arg) {
  const int nu = NU > 0 ? NU : nu_arg;
  using G = VT<N1>;
  constexpr int N = G::n1(L);
  constexpr int NT = G::grp(L);
  T* xa = base + G::off(L);
  T* xb = xa + G::np(L);
  T* bl = xb + G::np(L);
  const T d = lv[L].d, e = lv[L].e, c = lv[L].c, wd = lv[L].wd;
  if constexpr (N <= 7 && NT == 32) {
    // this level and all below it in the registers of the one warp that runs them
    constexpr int S = N + 2;
    const int lane = threadIdx.x & 31;
    T b[N], x[N];
#pragma unroll
    for (int y = 0; y < N; ++y) b[y] = lane < N ? bl[(y + 1) * S + lane + 1] : T(0);
    wl_cycle<T, N>(b, x, lv, L, nu, lane);
#pragma unroll
    for (int y = 0; y < N; ++y)
      if (lane < N) xa[(y + 1) * S + lane + 1] = x[y];
    __syncwarp();
    return 0;
  } else if constexpr (N == 1) {
    if (threadIdx.x == 0) xa[4] = bl[4] / d;
    vt_sync<NT>();
    return 0;
  } else {
    int cur = 0;
    if (nu == 2) {
      vt_level_pass<T, N, NT, 1>(xb, xa, bl, d, e, c, wd);
      vt_sync<NT>();
    } else {
      for (int q = threadIdx.x; q < G::np(L); q += NT) xa[q] = T(0);
      vt_sync<NT>();
      for (int sw = 0; sw < nu; ++sw) {
        if (cur == 0) vt_level_pass<T, N, NT, 0>(xa, xb, bl, d, e, c, wd);
        else vt_level_pass<T, N, NT, 0>(xb, xa, bl, d, e, c, wd);
        cur ^= 1;
        vt_sync<NT>();
      }
    }
    T* xcur = cur == 0 ? xa : xb;
    T* rbuf = cur == 0 ? xb : xa;
    vt_level_pass<T, N, NT, 2>(xcur, rbuf, bl, d, e, c, wd);
    vt_sync<NT>();
    T* bc = base + G::off(L + 1) + 2 * G::np(L + 1);
    vt_restrict<T, N, NT>(rbuf, bc);
    vt_sync<NT>();
    int ccur = 0;
    if (threadIdx.x < G::grp(L + 1)) ccur = vt_coarse<T, N1, L + 1, NU>(base, lv, nu);
    vt_sync<NT>();
    // the coarse result's buffer index is the same in every thread of the coarse group; share it
    __shared__ int cbuf;
    if (threadIdx.x == 0) cbuf = ccur;
    vt_sync<NT>();
    const T* xc = base + G::off(L + 1) + (cbuf == 0 ? 0 : G::np(L + 1));
    int sw0 = 0;
    if constexpr (CStrip<N, NT>::use && kVtFuseProlong<T>) {
      if (nu >= 1) {                                 // prolongation folded into the first sweep
        if (cur == 0) vt_cstrip<T, N, NT, 0, true>(xa, xb, bl, xc, d, e, c, wd);
        else vt_cstrip<T, N, NT, 0, true>(xb, xa, bl, xc, d, e, c, wd);
        cur ^= 1;
        vt_sync<NT>();
        sw0 = 1;
      }
    }
    if (sw0 == 0) {
      vt_prolong<T, N, NT>(xc, xcur);
      vt_sync<NT>();
    }
    for (int sw = sw0; sw < nu; ++sw) {
      if (cur == 0) vt_level_pass<T, N, NT, 0>(xa, xb, bl, d, e, c, wd);
      else vt_level_pass<T, N, NT, 0>(xb, xa, bl, d, e, c, wd);
      cur ^= 1;
      vt_sync<NT>();
    }
    return cur;
  }
}

// Level-0 sweeps of the V-cycle kernel.  Scalar form: a thread owns a strip of
// up to kStripRows rows of one grid column (vt_strip).  Float32 forms: a thread
// owns two columns over 8 rows and computes both nodes with packed FP32x2
// arithmetic (the same operations in the same order as vt_strip, per lane); the
// two columns are adjacent (four loads per row for the pair) or half a grid apart
// (six loads per row, but neighbouring lanes read neighbouring words).
template <typename T, int N1, bool PAIR = (std::is_same<T, float>::value && N1 >= 63)>
struct VtLevel0 {
  Strip g;
  T bv[kStripRows];
  __device__ __forceinline__ void init(const T* __restrict__ b0) {
    g = strip_of(N1);
#pragma unroll
    for (int j = 0; j < kStripRows; ++j) {
      const int y = g.y0 + j;
      bv[j] = (g.x >= 0 && y < g.y1) ? b0[y * N1 + g.x] : T(0);
    }
  }
  template <int MODE>
  __device__ __forceinline__ void pass(const T* __restrict__ xs, T* __restrict__ xd, T d, T e, T c, T wd) const {
    vt_strip<T, N1 + 2, MODE>(xs, xd, bv, g, d, e, c, wd);
  }
  template <bool PRO, bool OUT>
  __device__ __forceinline__ void post(const T* __restrict__ xs, T* __restrict__ xd, const T* __restrict__ xc,
                                       T* __restrict__ gout, bool acc, T d, T e, T c, T wd) const {
    vt_strip_post<T, N1, PRO, OUT>(xs, xd, xc, gout, acc, bv, g, d, e, c, wd);
  }
  __device__ __forceinline__ T first_b() const { return bv[0]; }
};

template <int N1>
struct VtLevel0<float, N1, true> {
  static constexpr int NP = (N1 + 1) / 2;      // column pairs (the last one has a single node)
  static constexpr int R = 8;                  // rows per thread
  static constexpr int S = N1 + 2;
  static_assert(VT<N1>::nb() / NP * R >= N1, "pair strips must cover the grid");
  int x0, y0, ny;
  bool v1;                                      // the pair's second node exists
  float2 bv[R];
  __device__ __forceinline__ void init(const float* __restrict__ b0) {
    const int t = threadIdx.x;
    const int px = t % NP, chunk = t / NP;
    x0 = 2 * px;
    y0 = chunk * R;
    ny = max(0, min(R, N1 - y0));
    v1 = x0 + 1 < N1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int y = y0 + j;
      bv[j] = j < ny ? make_float2(b0[y * N1 + x0], v1 ? b0[y * N1 + x0 + 1] : 0.f) : make_float2(0.f, 0.f);
    }
  }
  template <int MODE>
  __device__ __forceinline__ void pass(const float* __restrict__ xs, float* __restrict__ xd, float d, float e,
                                       float c, float wd) const {
    if (ny <= 0) return;
    float* q = xd + (y0 + 1) * S + x0 + 1;
    if (MODE == 1) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < ny) {
          q[j * S] = wd * bv[j].x;
          if (v1) q[j * S + 1] = wd * bv[j].y;
        }
      return;
    }
    const float* p = xs + y0 * S + x0;         // row y0 - 1, column x0 - 1 (zero-bordered)
    float a0 = p[0], b0 = p[1], c0 = p[2], d0 = v1 ? p[3] : 0.f;
    float a1 = p[S], b1 = p[S + 1], c1 = p[S + 2], d1 = v1 ? p[S + 3] : 0.f;
    const float2 dd = make_float2(d, d), ee = make_float2(e, e), cc = make_float2(c, c);
    const float2 ww = make_float2(wd, wd), m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (j < ny) {
        const float* pr = p + (j + 2) * S;
        const float a2 = pr[0], b2 = pr[1], c2 = pr[2], d2 = v1 ? pr[3] : 0.f;
        const float2 C = make_float2(b1, c1);
        const float2 edges = __fadd2_rn(__fadd2_rn(make_float2(b0, c0), make_float2(b2, c2)),
                                        __fadd2_rn(make_float2(a1, b1), make_float2(c1, d1)));
        const float2 corners = __fadd2_rn(__fadd2_rn(make_float2(a0, b0), make_float2(c0, d0)),
                                          __fadd2_rn(make_float2(a2, b2), make_float2(c2, d2)));
        const float2 av = __ffma2_rn(dd, C, __ffma2_rn(ee, edges, __fmul2_rn(cc, corners)));
        const float2 r = __ffma2_rn(m1, av, bv[j]);                 // b - A x, rounded once
        const float2 o = MODE == 2 ? r : __ffma2_rn(ww, r, C);
        q[j * S] = o.x;
        if (v1) q[j * S + 1] = o.y;
        a0 = a1; b0 = b1; c0 = c1; d0 = d1;
        a1 = a2; b1 = b2; c1 = c2; d1 = d2;
      }
    }
  }
  // post-smoothing sweep with the prolongation (PRO) or the copy-out (OUT) folded
  // in, as vt_strip_post.  Window columns (a, b, c, d) are the 1-based fine columns
  // x0 .. x0+3 (x0 even): their coarse column pairs are (A,A), (A,B), (B,B), (B,C)
  // with A = x0/2; window row w is fine row y0 + w (y0 even).
  template <bool PRO, bool OUT>
  __device__ __forceinline__ void post(const float* __restrict__ xs, float* __restrict__ xd,
                                       const float* __restrict__ xc, float* __restrict__ gout, bool acc, float d,
                                       float e, float c, float wd) const {
    if (ny <= 0) return;
    constexpr int SC = (N1 - 1) / 2 + 2;
    const float* p = xs + y0 * S + x0;
    const float* cp = xc + (y0 / 2) * SC + x0 / 2;
    const float2 q4 = make_float2(0.25f, 0.25f);
    float2 s01 = make_float2(0.f, 0.f), s23 = s01;     // pair sums of the last coarse row read
    auto csum = [&](int i, float2& u01, float2& u23) {
      const float* r = cp + i * SC;
      const float A = r[0], B = r[1], C = v1 ? r[2] : 0.f;
      u01 = __fadd2_rn(make_float2(A, A), make_float2(A, B));
      u23 = __fadd2_rn(make_float2(B, B), make_float2(B, C));
    };
    auto wrow = [&](int w, float& wa, float& wb, float& wc, float& wdn) {
      const float* pr = p + w * S;
      wa = pr[0]; wb = pr[1]; wc = pr[2]; wdn = v1 ? pr[3] : 0.f;
      if (PRO) {
        float2 k01, k23;
        if (w & 1) {
          float2 n01, n23;
          csum((w + 1) >> 1, n01, n23);
          k01 = __fmul2_rn(q4, __fadd2_rn(s01, n01));
          k23 = __fmul2_rn(q4, __fadd2_rn(s23, n23));
          s01 = n01; s23 = n23;
        } else {
          k01 = __fmul2_rn(q4, __fadd2_rn(s01, s01));
          k23 = __fmul2_rn(q4, __fadd2_rn(s23, s23));
        }
        const float2 ab = __fadd2_rn(make_float2(wa, wb), k01);
        const float2 cd = __fadd2_rn(make_float2(wc, wdn), k23);
        wa = ab.x; wb = ab.y; wc = cd.x; wdn = v1 ? cd.y : 0.f;
      }
    };
    float* q = xd + (y0 + 1) * S + x0 + 1;
    float* go = gout + y0 * N1 + x0;
    // the accumulator's values are all requested before the sweep, not one latency a row
    float2 ga[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
      ga[j] = (OUT && acc && j < ny) ? make_float2(go[j * N1], v1 ? go[j * N1 + 1] : 0.f) : make_float2(0.f, 0.f);
    if (PRO) csum(0, s01, s23);
    float a0, b0, c0, d0, a1, b1, c1, d1;
    wrow(0, a0, b0, c0, d0);
    wrow(1, a1, b1, c1, d1);
    const float2 dd = make_float2(d, d), ee = make_float2(e, e), cc = make_float2(c, c);
    const float2 ww = make_float2(wd, wd), m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (j < ny) {
        float a2, b2, c2, d2;
        wrow(j + 2, a2, b2, c2, d2);
        const float2 C = make_float2(b1, c1);
        const float2 edges = __fadd2_rn(__fadd2_rn(make_float2(b0, c0), make_float2(b2, c2)),
                                        __fadd2_rn(make_float2(a1, b1), make_float2(c1, d1)));
        const float2 corners = __fadd2_rn(__fadd2_rn(make_float2(a0, b0), make_float2(c0, d0)),
                                          __fadd2_rn(make_float2(a2, b2), make_float2(c2, d2)));
        const float2 av = __ffma2_rn(dd, C, __ffma2_rn(ee, edges, __fmul2_rn(cc, corners)));
        const float2 o = __ffma2_rn(ww, __ffma2_rn(m1, av, bv[j]), C);
        if (!OUT) {
          q[j * S] = o.x;
          if (v1) q[j * S + 1] = o.y;
        } else if (acc) {
          go[j * N1] = ga[j].x + o.x;
          if (v1) go[j * N1 + 1] = ga[j].y + o.y;
        } else {
          go[j * N1] = o.x;
          if (v1) go[j * N1 + 1] = o.y;
        }
        a0 = a1; b0 = b1; c0 = c1; d0 = d1;
        a1 = a2; b1 = b2; c1 = c2; d1 = d2;
      }
    }
  }
  __device__ __forceinline__ float first_b() const { return bv[0].x; }
};

template <int N1>
struct VtLevel0Split {
  // a thread owns grid columns xa and xa + NP over R rows: neighbouring lanes hold
  // neighbouring columns, so every shared-memory access of a warp is conflict-free
  static constexpr int NP = (N1 + 1) / 2;
  static constexpr int R = 8;                  // rows per thread
  static constexpr int S = N1 + 2;
  static_assert(VT<N1>::nb() / NP * R >= N1, "strips must cover the grid");
  static_assert(NP % 2 == 0, "the two columns of a thread must have the same parity");
  int xa, y0, ny;
  bool v1;                                      // the second column exists
  float2 bv[R];
  __device__ __forceinline__ void init(const float* __restrict__ b0) {
    const int t = threadIdx.x;
    xa = t % NP;
    y0 = (t / NP) * R;
    ny = max(0, min(R, N1 - y0));
    v1 = xa + NP < N1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int y = y0 + j;
      bv[j] = j < ny ? make_float2(b0[y * N1 + xa], v1 ? b0[y * N1 + xa + NP] : 0.f) : make_float2(0.f, 0.f);
    }
  }
  // window row of the two columns: left, centre, right neighbours as (column a, column b)
  __device__ __forceinline__ void wload(const float* pr, float2& l, float2& m, float2& r) const {
    l = make_float2(pr[0], v1 ? pr[NP] : 0.f);
    m = make_float2(pr[1], v1 ? pr[NP + 1] : 0.f);
    r = make_float2(pr[2], v1 ? pr[NP + 2] : 0.f);
  }
  template <int MODE>
  __device__ __forceinline__ void pass(const float* __restrict__ xs, float* __restrict__ xd, float d, float e,
                                       float c, float wd) const {
    if (ny <= 0) return;
    float* q = xd + (y0 + 1) * S + xa + 1;
    if (MODE == 1) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < ny) {
          q[j * S] = wd * bv[j].x;
          if (v1) q[j * S + NP] = wd * bv[j].y;
        }
      return;
    }
    const float* p = xs + y0 * S + xa;         // row y0 - 1, column xa - 1 (zero-bordered)
    float2 l0, m0, r0, l1, m1_, r1;
    wload(p, l0, m0, r0);
    wload(p + S, l1, m1_, r1);
    const float2 dd = make_float2(d, d), ee = make_float2(e, e), cc = make_float2(c, c);
    const float2 ww = make_float2(wd, wd), neg = make_float2(-1.f, -1.f);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (j < ny) {
        float2 l2, m2, r2;
        wload(p + (j + 2) * S, l2, m2, r2);
        const float2 edges = __fadd2_rn(__fadd2_rn(m0, m2), __fadd2_rn(l1, r1));
        const float2 corners = __fadd2_rn(__fadd2_rn(l0, r0), __fadd2_rn(l2, r2));
        const float2 av = __ffma2_rn(dd, m1_, __ffma2_rn(ee, edges, __fmul2_rn(cc, corners)));
        const float2 rr = __ffma2_rn(neg, av, bv[j]);                // b - A x, rounded once
        const float2 o = MODE == 2 ? rr : __ffma2_rn(ww, rr, m1_);
        q[j * S] = o.x;
        if (v1) q[j * S + NP] = o.y;
        l0 = l1; m0 = m1_; r0 = r1;
        l1 = l2; m1_ = m2; r1 = r2;
      }
    }
  }
  // post-smoothing sweep with the prolongation (PRO) or the copy-out (OUT) folded
  // in, as vt_strip_post; both columns have the parity of xa, so the coarse pair
  // sums of a window row are formed by the same selects for both
  template <bool PRO, bool OUT>
  __device__ __forceinline__ void post(const float* __restrict__ xs, float* __restrict__ xd,
                                       const float* __restrict__ xc, float* __restrict__ gout, bool acc, float d,
                                       float e, float c, float wd) const {
    if (ny <= 0) return;
    constexpr int SC = (N1 - 1) / 2 + 2;
    const float* p = xs + y0 * S + xa;
    const int lo = xa >> 1;
    const bool odd = xa & 1;
    const float* cp = xc + (y0 / 2) * SC + lo;
    const float2 q4 = make_float2(0.25f, 0.25f);
    float2 s0[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    auto csum = [&](int i, float2 (&sv)[3]) {
      const float* qa = cp + i * SC;
      const float* qb = qa + NP / 2;
      const float2 v0 = make_float2(qa[0], v1 ? qb[0] : 0.f);
      const float2 w1 = make_float2(qa[1], v1 ? qb[1] : 0.f);
      const float2 v2 = odd ? make_float2(qa[2], v1 ? qb[2] : 0.f) : make_float2(0.f, 0.f);
      const float2 m0 = odd ? w1 : v0;
      sv[0] = __fadd2_rn(v0, m0);
      sv[1] = __fadd2_rn(m0, w1);
      sv[2] = __fadd2_rn(w1, odd ? v2 : w1);
    };
    auto wrow = [&](int w, float2& l, float2& m, float2& r) {
      wload(p + w * S, l, m, r);
      if (PRO) {
        float2 k[3];
        if (w & 1) {
          float2 s1[3];
          csum((w + 1) >> 1, s1);
#pragma unroll
          for (int q = 0; q < 3; ++q) { k[q] = __fmul2_rn(q4, __fadd2_rn(s0[q], s1[q])); s0[q] = s1[q]; }
        } else {
#pragma unroll
          for (int q = 0; q < 3; ++q) k[q] = __fmul2_rn(q4, __fadd2_rn(s0[q], s0[q]));
        }
        l = __fadd2_rn(l, k[0]);
        m = __fadd2_rn(m, k[1]);
        r = __fadd2_rn(r, k[2]);
      }
    };
    float* q = xd + (y0 + 1) * S + xa + 1;
    float* go = gout + y0 * N1 + xa;
    // the accumulator's values are all requested before the sweep, not one latency a row
    float2 ga[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
      ga[j] = (OUT && acc && j < ny) ? make_float2(go[j * N1], v1 ? go[j * N1 + NP] : 0.f) : make_float2(0.f, 0.f);
    if (PRO) csum(0, s0);
    float2 l0, m0, r0, l1, m1_, r1;
    wrow(0, l0, m0, r0);
    wrow(1, l1, m1_, r1);
    const float2 dd = make_float2(d, d), ee = make_float2(e, e), cc = make_float2(c, c);
    const float2 ww = make_float2(wd, wd), neg = make_float2(-1.f, -1.f);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (j < ny) {
        float2 l2, m2, r2;
        wrow(j + 2, l2, m2, r2);
        const float2 edges = __fadd2_rn(__fadd2_rn(m0, m2), __fadd2_rn(l1, r1));
        const float2 corners = __fadd2_rn(__fadd2_rn(l0, r0), __fadd2_rn(l2, r2));
        const float2 av = __ffma2_rn(dd, m1_, __ffma2_rn(ee, edges, __fmul2_rn(cc, corners)));
        const float2 o = __ffma2_rn(ww, __ffma2_rn(neg, av, bv[j]), m1_);
        if (!OUT) {
          q[j * S] = o.x;
          if (v1) q[j * S + NP] = o.y;
        } else if (acc) {
          go[j * N1] = ga[j].x + o.x;
          if (v1) go[j * N1 + NP] = ga[j].y + o.y;
        } else {
          go[j * N1] = o.x;
          if (v1) go[j * N1 + NP] = o.y;
        }
        l0 = l1; m0 = m1_; r0 = r1;
        l1 = l2; m1_ = m2; r1 = r2;
      }
    }
  }
  __device__ __forceinline__ float first_b() const { return bv[0].x; }
};

// the level-0 form a kernel uses: split column pairs at 127 x 127 (32 warps, where the
// bank conflicts of adjacent pairs dominate), adjacent pairs at 63 x 63 (8 warps, where
// the fewer loads of adjacent pairs win), scalar strips otherwise
template <typename T, int N1>
using VtLevel0Of = typename std::conditional<std::is_same<T, float>::value && N1 >= 127, VtLevel0Split<N1>,
                                             VtLevel0<T, N1>>::type;

template <typename T, int N1, int NU>
__global__ void __launch_bounds__(VT<N1>::nb(), sizeof(T) == 8 && N1 < 127 ? 2 : kVFThreads / VT<N1>::nb()) vcycle_t_kernel(const T* __restrict__ bg, T* xg, FusedLevels L,
                                                                 T omega, int nu_arg, T* acc, int64_t acc_ss, int acc_L,
                                                                 int acc_col0, VColumns cols, const VtMulti vm) {
  using G = VT<N1>;
  constexpr int NL = G::nlev();
  constexpr int S0 = N1 + 2;
  // smoothing sweeps: fixed at compile time in the NU > 0 instantiation (no code for other counts)
  const int nu = NU > 0 ? NU : nu_arg;
  extern __shared__ __align__(32) unsigned char vt_smem_raw[];
  __shared__ VFLevel<T> lv[13];
  T* base = reinterpret_cast<T*>(vt_smem_raw);
  int64_t col = blockIdx.x;
  // member of a merged launch: columns [g*per, (g+1)*per) belong to member g, whose
  // right-hand sides, outputs and level stencils replace those of the shared arguments
  int g = 0;
  if (vm.ng > 1) {
    g = int(col / vm.per);
    col -= int64_t(g) * vm.per;
#pragma unroll
    for (int i = 1; i < kMaxGroup; ++i) {
      if (i == g) {
        bg = static_cast<const T*>(vm.b[i]); xg = static_cast<T*>(vm.x[i]); acc = static_cast<T*>(vm.acc[i]);
      }
    }
  }
  constexpr int n0 = N1 * N1;
  // the column's right-hand side, and its output: x itself, or the strided column x is
  // added to (or stored into)
  const T* bcol = cols.b_L > 0 ? bg + (col / cols.b_L) * cols.b_ss + (col % cols.b_L) * int64_t(n0) : bg + col * n0;
  const bool acc_on = acc != nullptr && cols.acc_add;
  T* gout = acc != nullptr ? acc + (col / acc_L) * acc_ss + (acc_col0 + col % acc_L) * int64_t(n0) : xg + col * n0;
  // level constants, by the last warp (which has the least border work)
  if (threadIdx.x >= G::nb() - 32 && threadIdx.x < G::nb() - 32 + NL) {
    const int l = threadIdx.x - (G::nb() - 32);
    const double dd = g == 0 ? L.diag[l] : vm.diag[g][l];
    const double de = g == 0 ? L.edge[l] : vm.edge[g][l];
    const double dc = g == 0 ? L.corner[l] : vm.corner[g][l];
    lv[l].d = T(dd); lv[l].e = T(de); lv[l].c = T(dc);
    lv[l].wd = omega / T(dd);
  }
  // zero borders of every array (interiors are always written before they are read):
  // border thread k of an s x s array zeroes position k of its four sides
  for (int t0 = threadIdx.x; t0 < G::border_threads(); t0 += G::nb()) {
    int t = t0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int s = G::s(l), narr = l > 0 ? 3 : 2;
      if (t >= 0 && t < narr * s) {
        const int arr = t / s, k = t - arr * s;
        T* A = base + G::off(l) + arr * s * s;
        A[k] = T(0);
        A[(s - 1) * s + k] = T(0);
        A[k * s] = T(0);
        A[k * s + s - 1] = T(0);
      }
      t -= narr * s;
    }
  }
  pdl_wait();                                        // b and the output are shared with earlier kernels
  VtLevel0Of<T, N1> z;
  z.init(bcol);
  __syncthreads();
  T* xa = base;
  T* xb = base + G::np(0);
  int cur = 0;
  if constexpr (N1 == 1) {
    if (threadIdx.x == 0) xa[4] = z.first_b() / lv[0].d;
    __syncthreads();
  } else {
    constexpr int NT0 = G::grp(0);
    const T d = lv[0].d, e = lv[0].e, c = lv[0].c, wd = lv[0].wd;
    if (threadIdx.x < NT0) {
      if (nu == 0) {
        for (int q = threadIdx.x; q < G::np(0); q += NT0) xa[q] = T(0);
        vt_sync<NT0>();
      }
      for (int sw = 0; sw < nu; ++sw) {
        if (sw == 0) z.template pass<1>(xb, xa, d, e, c, wd);
        else if (cur == 0) z.template pass<0>(xa, xb, d, e, c, wd);
        else z.template pass<0>(xb, xa, d, e, c, wd);
        cur = sw == 0 ? 0 : cur ^ 1;
        vt_sync<NT0>();
      }
      T* xcur = cur == 0 ? xa : xb;
      T* rbuf = cur == 0 ? xb : xa;
      z.template pass<2>(xcur, rbuf, d, e, c, wd);
      vt_sync<NT0>();
      vt_restrict<T, N1, NT0>(rbuf, base + G::off(1) + 2 * G::np(1));
      vt_sync<NT0>();
      int ccur = 0;
      if (threadIdx.x < G::grp(1)) ccur = vt_coarse<T, N1, 1, NU>(base, lv, nu);
      vt_sync<NT0>();
      __shared__ int cbuf0;
      if (threadIdx.x == 0) cbuf0 = ccur;
      vt_sync<NT0>();
      const T* xc = base + G::off(1) + (cbuf0 == 0 ? 0 : G::np(1));
      pdl_trigger();                                   // only the post-smoothing and the write remain
      // the copy-out is folded into the last sweep; in float32 the prolongation
      // into the first (in float64 the extra window corrections cost more than the pass)
      int sw0 = 0;
      if constexpr (kVtFuseProlong<T>) {
        if (nu >= 2) {
          z.template post<true, false>(xa + cur * G::np(0), xa + (cur ^ 1) * G::np(0), xc, gout, acc_on, d, e, c, wd);
          cur ^= 1;
          vt_sync<NT0>();
          sw0 = 1;
        }
      }
      if (sw0 == 0) {
        vt_prolong<T, N1, NT0>(xc, xcur);
        vt_sync<NT0>();
      }
      if (nu >= 1) {
        for (int sw = sw0; sw + 1 < nu; ++sw) {
          if (cur == 0) z.template pass<0>(xa, xb, d, e, c, wd); else z.template pass<0>(xb, xa, d, e, c, wd);
          cur ^= 1;
          vt_sync<NT0>();
        }
        z.template post<false, true>(xa + cur * G::np(0), xa + (cur ^ 1) * G::np(0), xc, gout, acc_on, d, e, c, wd);
      }
    } else {
      pdl_trigger();
    }
    if (nu >= 1) return;                               // the last sweep wrote the column
    __syncthreads();
  }
  if constexpr (N1 == 1) pdl_trigger();
  __shared__ int cfin;
  if (threadIdx.x == 0) cfin = cur;
  __syncthreads();
  const T* x0 = base + (cfin == 0 ? 0 : G::np(0));
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (acc_on) {
    for (int y = ty; y < N1; y += G::nb() / 32)
      for (int x = tx; x < N1; x += 32) gout[y * N1 + x] += x0[(y + 1) * S0 + x + 1];
  } else {
    for (int y = ty; y < N1; y += G::nb() / 32)
      for (int x = tx; x < N1; x += 32) gout[y * N1 + x] = x0[(y + 1) * S0 + x + 1];
  }
}

template <typename T, int N1>
static cudaError_t launch_vt(const T* b, T* x, int64_t B, const FusedLevels& L, T omega, int nu, T* acc,
                             int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st, VColumns cols,
                             const VtMulti& vm) {
  const size_t smem = size_t(VT<N1>::total()) * sizeof(T);
  // V(2,2), the cycle of every solve, has an instantiation of its own; other sweep counts share one
  auto k = nu == 2 ? vcycle_t_kernel<T, N1, 2> : vcycle_t_kernel<T, N1, 0>;
  cudaError_t e = allow_max_smem(k);
  if (e != cudaSuccess) return e;
  {
    const cudaError_t le_ = launch_pdl(k, (dim3(unsigned(B * vm.ng))), dim3(VT<N1>::nb()), size_t(smem), st,
                                      b, x, L, omega, nu, acc, acc_ss, acc_L, acc_col0, cols, vm);
    if (le_ != cudaSuccess) return le_;
  }
  return cudaGetLastError();
}

size_t vcycle_full_smem(const FusedLevels& L, int esize) {
  size_t s = 0;
  for (int l = 0; l < L.nlev; ++l) s += size_t(L.n1[l] + 2) * (L.n1[l] + 2) * (l > 0 ? 3 : 2) * esize;
  return s;
}

bool vcycle_full_fits(const FusedLevels& L, int esize) {
  const int n1 = L.n1[0];
  const int nchunks = (n1 + kStripRows - 1) / kStripRows;
  const int nb = n1 >= 127 ? kVFThreads : 256;          // threads of the instantiation for this top level
  return int64_t(nchunks) * n1 <= nb && vcycle_full_smem(L, esize) <= kMaxSmem;
}

template <typename T>
static cudaError_t launch_vt_any(const T* b, T* x, int64_t B, const FusedLevels& L, T omega, int nu, T* acc,
                                 int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st, VColumns cols,
                                 const VtMulti& vm) {
  if (B == 0) return cudaSuccess;
  if (!vcycle_full_fits(L, sizeof(T))) return cudaErrorInvalidConfiguration;
  const double n0 = double(L.n1[0]) * L.n1[0];
  ProfScope ps(KK_VCYCLE_FUSED, st, double(sizeof(T)) * B * vm.ng * n0 * (acc ? 3 : 2),
               double(B) * vm.ng * n0 * (4.0 / 3.0) * (21.0 * 2 * nu + 18.0 + 10.0));
  cudaError_t e;
  switch (L.n1[0]) {
    case 1: e = launch_vt<T, 1>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    case 3: e = launch_vt<T, 3>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    case 7: e = launch_vt<T, 7>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    case 15: e = launch_vt<T, 15>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    case 31: e = launch_vt<T, 31>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    case 63: e = launch_vt<T, 63>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    case 127: e = launch_vt<T, 127>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, vm); break;
    default: return cudaErrorInvalidConfiguration;
  }
  note_launch();
  return e;
}

template <typename T>
cudaError_t launch_vcycle_full(const T* b, T* x, int64_t B, const FusedLevels& L, T omega, int nu, T* acc,
                               int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st, VColumns cols) {
  static const VtMulti solo{};
  return launch_vt_any<T>(b, x, B, L, omega, nu, acc, acc_ss, acc_L, acc_col0, st, cols, solo);
}

template <typename T>
cudaError_t launch_vcycle_full_group(const T* const* b, T* const* x, T* const* acc, const FusedLevels* L, int ng,
                                     int64_t B, T omega, int nu, int64_t acc_ss, int acc_L, int acc_col0,
                                     cudaStream_t st, VColumns cols) {
  if (ng < 1 || ng > kMaxGroup) return cudaErrorInvalidValue;
  VtMulti vm{};
  vm.ng = ng;
  vm.per = B;
  for (int g = 0; g < ng; ++g) {
    if (L[g].nlev != L[0].nlev || L[g].n1[0] != L[0].n1[0]) return cudaErrorInvalidValue;
    if ((acc[g] != nullptr) != (acc[0] != nullptr)) return cudaErrorInvalidValue;
    vm.b[g] = b[g]; vm.x[g] = x[g]; vm.acc[g] = acc[g];
    for (int l = 0; l < L[g].nlev; ++l) {
      vm.diag[g][l] = L[g].diag[l]; vm.edge[g][l] = L[g].edge[l]; vm.corner[g][l] = L[g].corner[l];
    }
  }
  return launch_vt_any<T>(b[0], x[0], B, L[0], omega, nu, acc[0], acc_ss, acc_L, acc_col0, st, cols, vm);
}

// ---------------------------------------------------------------------------
// Cluster V-cycle: one thread-block cluster of C CTAs per column.  The fine
// levels ("distributed", band height B_l = (n1_l + 1) / C of at least 8 rows)
// are split into horizontal bands, one per CTA; each band array carries one
// halo row above and below, filled from the neighbouring CTAs' shared memory
// (DSMEM) after a cluster barrier whenever a pass reads neighbours.  The first
// level below the distributed ones is gathered into every CTA, and the
// remaining small levels are solved redundantly (identically) in each CTA.
// Local band row i of rank r holds global row r*B + i - 1; the last rank's
// row B is the Dirichlet boundary and stays zero.
// ---------------------------------------------------------------------------
constexpr int kVCThreads = 512;
constexpr int kCStrip = 16;

template <typename T>
struct VCLevel { int off, n1, band, rows, s; T d, e, c, wd; };

template <typename T, int MODE>   // 0 jacobi, 1 from zero, 2 residual; b in smem (band layout)
__device__ __forceinline__ void band_pass(const T* __restrict__ xs, T* __restrict__ xd, const T* __restrict__ b,
                                         int rows, int n1, int s, T d, T e, T c, T wd) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = 1 + ty; i <= rows; i += kVCThreads / 32)
    for (int x = tx; x < n1; x += 32) {
      const int o = i * s + x + 1;
      if (MODE == 1) { xd[o] = wd * b[o]; continue; }
      const T edges = (xs[o - s] + xs[o + s]) + (xs[o - 1] + xs[o + 1]);
      const T corners = (xs[o - s - 1] + xs[o - s + 1]) + (xs[o + s - 1] + xs[o + s + 1]);
      const T r = b[o] - fma(d, xs[o], fma(e, edges, c * corners));
      xd[o] = MODE == 2 ? r : fma(wd, r, xs[o]);
    }
}

// level-0 strip pass with the right-hand side in registers (strip of `cr` rows)
template <typename T, int MODE>
__device__ __forceinline__ void cstrip_pass(const T* __restrict__ xs, T* __restrict__ xd, const T (&bv)[kCStrip],
                                           int x, int i0, int cr, int s, T d, T e, T c, T wd) {
  if (x < 0) return;
  if (MODE == 1) {
#pragma unroll
    for (int j = 0; j < kCStrip; ++j)
      if (j < cr) xd[(i0 + j) * s + x + 1] = wd * bv[j];
    return;
  }
  const T* p = xs + (i0 - 1) * s + x;
  T wm0 = p[0], wc0 = p[1], wp0 = p[2];
  p += s;
  T wm1 = p[0], wc1 = p[1], wp1 = p[2];
  T* q = xd + i0 * s + x + 1;
#pragma unroll
  for (int j = 0; j < kCStrip; ++j) {
    if (j < cr) {
      p += s;
      const T wm2 = p[0], wc2 = p[1], wp2 = p[2];
      const T edges = (wc0 + wc2) + (wm1 + wp1);
      const T corners = (wm0 + wp0) + (wm2 + wp2);
      const T r = bv[j] - fma(d, wc1, fma(e, edges, c * corners));
      *q = MODE == 2 ? r : fma(wd, r, wc1);
      q += s;
      wm0 = wm1; wc0 = wc1; wp0 = wp1;
      wm1 = wm2; wc1 = wc2; wp1 = wp2;
    }
  }
}

// fill the halo rows of band array X from the neighbouring CTAs (caller: cluster.sync() before)
template <typename T>
__device__ __forceinline__ void band_exchange(T* X, int band, int s, int rank, int C) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  if (rank > 0) {
    const T* up = cl.map_shared_rank(X, rank - 1);
    for (int q = threadIdx.x; q < s; q += kVCThreads) X[q] = up[band * s + q];
  }
  if (rank < C - 1) {
    const T* dn = cl.map_shared_rank(X, rank + 1);
    for (int q = threadIdx.x; q < s; q += kVCThreads) X[(band + 1) * s + q] = dn[s + q];
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kVCThreads) vcycle_cluster_kernel(const T* __restrict__ bg, T* xg,
                                                                    ClusterLevels L, T omega, int nu, T* acc,
                                                                    int64_t acc_ss, int acc_L, int acc_col0) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(32) unsigned char vc_smem_raw[];
  __shared__ VCLevel<T> lv[13];
  __shared__ int curs[13];
  T* base = reinterpret_cast<T*>(vc_smem_raw);
  const int C = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const int64_t col = blockIdx.x / C;
  const int nlev = L.nlev, nd = L.nd;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int l = 0; l < nlev; ++l) {
      const int n1 = L.n1[l], s = n1 + 2;
      lv[l].n1 = n1; lv[l].s = s; lv[l].off = o;
      if (l < nd) {
        const int band = (n1 + 1) / C;
        lv[l].band = band;
        lv[l].rows = min(band, n1 - rank * band);          // valid rows of this rank
        o += (band + 2) * s * (l > 0 ? 3 : 2);
      } else {
        lv[l].band = n1; lv[l].rows = n1;
        o += s * s * 3;
      }
      lv[l].d = T(L.diag[l]); lv[l].e = T(L.edge[l]); lv[l].c = T(L.corner[l]);
      lv[l].wd = omega / T(L.diag[l]);
    }
    curs[0] = o;                                           // total elements (used just below)
  }
  __syncthreads();
  for (int q = threadIdx.x; q < curs[0]; q += kVCThreads) base[q] = T(0);
  // level-0 strip geometry and right-hand side (registers)
  const VCLevel<T> L0 = lv[0];
  const int n10 = L0.n1;
  const int nch = max(1, min(kVCThreads / n10, (L0.rows + kCStrip - 1) / 1));
  const int cr = (L0.rows + nch - 1) / nch;               // rows per strip (<= kCStrip by construction)
  int sx = -1, si0 = 1, scr = 0;
  {
    const int t = threadIdx.x, ch = t / n10;
    if (ch < nch) {
      sx = t - ch * n10;
      si0 = 1 + ch * cr;
      scr = max(0, min(cr, L0.rows - ch * cr));
      if (scr == 0) sx = -1;
    }
  }
  pdl_wait();
  T bv[kCStrip];
  {
    const T* b0 = bg + col * int64_t(n10) * n10;
#pragma unroll
    for (int j = 0; j < kCStrip; ++j) {
      const int gy = rank * L0.band + si0 - 1 + j;
      bv[j] = (sx >= 0 && j < scr) ? b0[int64_t(gy) * n10 + sx] : T(0);
    }
  }
  cl.sync();                                                // zeroed everywhere before any exchange
  // ----- descent -----
#pragma unroll 1
  for (int l = 0; l < nlev - 1; ++l) {
    const VCLevel<T> P = lv[l];
    const VCLevel<T> Q = lv[l + 1];
    const bool dist = l < nd;
    const int s = P.s;
    const int hgt = dist ? P.band + 2 : P.n1 + 2;
    T* xa = base + P.off;
    T* xb = xa + hgt * s;
    const T* bl = xb + hgt * s;
    int cur = 0;
#pragma unroll 1
    for (int sw = 0; sw < nu; ++sw) {
      T* src = cur == 0 ? xa : xb;
      T* dst = sw == 0 ? xa : (cur == 0 ? xb : xa);
      if (sw > 0) {
        if (dist) { cl.sync(); band_exchange(src, P.band, s, rank, C); }
        else __syncthreads();
      }
      if (l == 0) {
        if (sw == 0) cstrip_pass<T, 1>(src, dst, bv, sx, si0, scr, s, P.d, P.e, P.c, P.wd);
        else cstrip_pass<T, 0>(src, dst, bv, sx, si0, scr, s, P.d, P.e, P.c, P.wd);
      } else {
        if (sw == 0) band_pass<T, 1>(src, dst, bl, P.rows, P.n1, s, P.d, P.e, P.c, P.wd);
        else band_pass<T, 0>(src, dst, bl, P.rows, P.n1, s, P.d, P.e, P.c, P.wd);
      }
      cur = dst == xa ? 0 : 1;
    }
    T* xcur = cur == 0 ? xa : xb;
    T* rbuf = cur == 0 ? xb : xa;
    if (dist) { cl.sync(); band_exchange(xcur, P.band, s, rank, C); }
    else __syncthreads();
    if (l == 0) cstrip_pass<T, 2>(xcur, rbuf, bv, sx, si0, scr, s, P.d, P.e, P.c, P.wd);
    else band_pass<T, 2>(xcur, rbuf, bl, P.rows, P.n1, s, P.d, P.e, P.c, P.wd);
    // restriction into the coarse right-hand side
    const int sc = Q.s;
    const bool cdist = (l + 1) < nd;
    T* bc = base + Q.off + 2 * (cdist ? Q.band + 2 : Q.n1 + 2) * sc;
    if (dist) { cl.sync(); band_exchange(rbuf, P.band, s, rank, C); }
    else __syncthreads();
    {
      const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
      // coarse rows handled here: local band rows (distributed coarse) or this rank's
      // global rows (first gathered level) or all rows (redundant)
      const int cb = dist ? P.band / 2 : 0;                    // coarse band height of this rank
      const int nrows = dist ? min(cb, Q.n1 - rank * cb) : Q.n1;
      for (int ic = ty; ic < nrows; ic += kVCThreads / 32) {
        // fine local row of the coarse row's centre: dist -> 2*ic + 2 (band layout), else 2*ic + 2 (padded)
        const T* r = rbuf + (2 * ic + 2) * s;
        T* out = cdist ? bc + (ic + 1) * sc : bc + (dist ? rank * cb + ic + 1 : ic + 1) * sc;
        for (int I = tx; I < Q.n1; I += 32) {
          const T* rr = r + 2 * I + 2;
          const T cen = rr[0];
          const T edg = (rr[s] + rr[-s]) + (rr[1] + rr[-1]);
          const T cor = (rr[s + 1] + rr[s - 1]) + (rr[-s + 1] + rr[-s - 1]);
          out[I + 1] = cen + T(0.5) * edg + T(0.25) * cor;
        }
      }
    }
    if (dist && !cdist) {
      // gather the first redundant level's right-hand side from every rank
      cl.sync();
      const int cb = P.band / 2;
      for (int rk = 0; rk < C; ++rk) {
        if (rk == rank) continue;
        const T* peer = cl.map_shared_rank(bc, rk);
        const int r0 = rk * cb, nr = min(cb, Q.n1 - r0);
        for (int q = threadIdx.x; q < nr * sc; q += kVCThreads) bc[(r0 + 1) * sc + q] = peer[(r0 + 1) * sc + q];
      }
    }
    if (threadIdx.x == 0) curs[l] = cur;
    __syncthreads();
  }
  // coarsest: one node (redundant in every CTA)
  if (threadIdx.x == 0) {
    const int l = nlev - 1;
    T* xa = base + lv[l].off;
    xa[4] = xa[2 * 9 + 4] / lv[l].d;
    curs[l] = 0;
  }
  __syncthreads();
  // ----- ascent -----
#pragma unroll 1
  for (int l = nlev - 2; l >= 0; --l) {
    const VCLevel<T> P = lv[l];
    const VCLevel<T> Q = lv[l + 1];
    const bool dist = l < nd, cdist = (l + 1) < nd;
    const int s = P.s, sc = Q.s;
    const int hgt = dist ? P.band + 2 : P.n1 + 2;
    const int hgtc = cdist ? Q.band + 2 : Q.n1 + 2;
    T* xa = base + P.off;
    T* xb = xa + hgt * s;
    const T* bl = xb + hgt * s;
    T* xca = base + Q.off;
    T* xc = curs[l + 1] == 0 ? xca : xca + hgtc * sc;
    if (cdist) { cl.sync(); band_exchange(xc, Q.band, sc, rank, C); }
    else __syncthreads();
    int cur = curs[l];
    {
      T* xf = cur == 0 ? xa : xb;
      const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
      const int rows = dist ? P.rows : P.n1;
      for (int i = 1 + ty; i <= rows; i += kVCThreads / 32) {
        // coarse local rows of fine local row i: distributed fine over distributed coarse ->
        // (i >> 1, (i + 1) >> 1); distributed fine over the full coarse grid -> global rows
        int c0, c1;
        if (!dist || cdist) { c0 = i >> 1; c1 = (i + 1) >> 1; }
        else { const int gi = rank * P.band + i; c0 = gi >> 1; c1 = (gi + 1) >> 1; }
        const T* r0 = xc + c0 * sc;
        const T* r1 = xc + c1 * sc;
        for (int x = tx; x < P.n1; x += 32) {
          const int gx = x + 1;
          const int a0 = gx >> 1, a1 = (gx + 1) >> 1;
          xf[i * s + x + 1] += T(0.25) * ((r0[a0] + r0[a1]) + (r1[a0] + r1[a1]));
        }
      }
    }
#pragma unroll 1
    for (int sw = 0; sw < nu; ++sw) {
      T* src = cur == 0 ? xa : xb;
      T* dst = cur == 0 ? xb : xa;
      if (dist) { cl.sync(); band_exchange(src, P.band, s, rank, C); }
      else __syncthreads();
      if (l == 0) cstrip_pass<T, 0>(src, dst, bv, sx, si0, scr, s, P.d, P.e, P.c, P.wd);
      else band_pass<T, 0>(src, dst, bl, P.rows, P.n1, s, P.d, P.e, P.c, P.wd);
      cur ^= 1;
    }
    if (threadIdx.x == 0) curs[l] = cur;
    __syncthreads();
  }
  pdl_trigger();
  // this rank's band of the level-0 result
  {
    const T* x0 = base + (curs[0] == 0 ? 0 : (L0.band + 2) * L0.s);
    const int s0 = L0.s;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n0 = int64_t(n10) * n10;
    T* dstg = acc ? acc + (col / acc_L) * acc_ss + (acc_col0 + col % acc_L) * n0 : xg + col * n0;
    for (int i = ty; i < L0.rows; i += kVCThreads / 32) {
      const int64_t gy = int64_t(rank) * L0.band + i;
      for (int x = tx; x < n10; x += 32) {
        const T v = x0[(i + 1) * s0 + x + 1];
        if (acc) dstg[gy * n10 + x] += v; else dstg[gy * n10 + x] = v;
      }
    }
  }
  cl.sync();                                               // peers may still read our shared memory
}

size_t vcycle_cluster_smem(const ClusterLevels& L, int C, int esize) {
  size_t o = 0;
  for (int l = 0; l < L.nlev; ++l) {
    const size_t s = L.n1[l] + 2;
    if (l < L.nd) o += (size_t((L.n1[l] + 1) / C) + 2) * s * (l > 0 ? 3 : 2);
    else o += s * s * 3;
  }
  return o * esize;
}

template <typename T>
cudaError_t launch_vcycle_cluster(const T* b, T* x, int64_t B, const ClusterLevels& L, int C, T omega, int nu, T* acc,
                                  int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const size_t smem = vcycle_cluster_smem(L, C, sizeof(T));
  if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
  cudaError_t e = allow_max_smem(vcycle_cluster_kernel<T>);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(vcycle_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(B * C));
  cfg.blockDim = dim3(kVCThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // cluster launches take full stream dependencies on both sides: with programmatic
  // overlap around this kernel, hGS results were wrong unless it triggered at once
  take_fence(st);
  const double n0 = double(L.n1[0]) * L.n1[0];
  ProfScope ps(KK_VCYCLE_FUSED, st, double(sizeof(T)) * B * n0 * (acc ? 3 : 2),
               double(B) * n0 * (4.0 / 3.0) * (21.0 * 2 * nu + 18.0 + 10.0));
  e = cudaLaunchKernelEx(&cfg, vcycle_cluster_kernel<T>, b, x, L, omega, nu, acc, acc_ss, acc_L, acc_col0);
  pdl_fence(st);
  note_launch();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic float64 reductions and MINRES recurrences
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ double block_sum(double v) {
  __shared__ double red[NT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;   // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(256) dot_kernel(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* partial) {
  pdl_enter();
  double s = 0.0;
  const int64_t stride = int64_t(kDotBlocks) * 256;
  int64_t i = blockIdx.x * int64_t(256) + threadIdx.x;
  // four strides' loads in flight before their (in-order) accumulation
  for (; i + 3 * stride < n; i += 4 * stride) {
    const T a0 = a[i], b0 = b[i], a1 = a[i + stride], b1 = b[i + stride];
    const T a2 = a[i + 2 * stride], b2 = b[i + 2 * stride], a3 = a[i + 3 * stride], b3 = b[i + 3 * stride];
    s = fma(double(a0), double(b0), s);
    s = fma(double(a1), double(b1), s);
    s = fma(double(a2), double(b2), s);
    s = fma(double(a3), double(b3), s);
  }
  for (; i < n; i += stride) s = fma(double(a[i]), double(b[i]), s);
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// float32 operands, float64-accurate inner product with little float64 work.
// GB300 executes float64 arithmetic at about 1/64 of the float32 rate, so one
// float64 FMA per entry would make the dot bound by the float64 pipe.  Instead
// every group of four entries is split exactly with error-free transformations
// in float32 (intrinsics, so nothing is contracted or reassociated):
//   TwoProduct: p = fl(x y), e = fma(x, y, -p)            => x y = p + e exactly
//   TwoSum:     s = fl(a + b), t = (a - (s - b')) + (b - b'), b' = s - a  => a + b = s + t exactly
// so that x.y over the group = s + (sum of the seven small error terms), exactly;
// s is accumulated in float64 (one float64 add per four entries) and the small
// terms, each below 2^-24 of the partial sums they come from, in float32.  The
// result is the float64 inner product up to a relative error of order 2^-48
// (against 2^-53 per add for float64 accumulation), deterministic (fixed order).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void dot4_exact(const float4& x, const float4& y, double& S, float& C) {
  const float p0 = __fmul_rn(x.x, y.x), p1 = __fmul_rn(x.y, y.y);
  const float p2 = __fmul_rn(x.z, y.z), p3 = __fmul_rn(x.w, y.w);
  const float e0 = __fmaf_rn(x.x, y.x, -p0), e1 = __fmaf_rn(x.y, y.y, -p1);
  const float e2 = __fmaf_rn(x.z, y.z, -p2), e3 = __fmaf_rn(x.w, y.w, -p3);
  float s01, t01, s23, t23, s, t;
  two_sum(p0, p1, s01, t01);
  two_sum(p2, p3, s23, t23);
  two_sum(s01, s23, s, t);
  S = __dadd_rn(S, double(s));
  C = __fadd_rn(C, __fadd_rn(__fadd_rn(__fadd_rn(t, t01), __fadd_rn(t23, e0)),
                             __fadd_rn(__fadd_rn(e1, e2), e3)));
}

__global__ void __launch_bounds__(256) dot4_kernel(const float4* __restrict__ a, const float4* __restrict__ b,
                                                   int64_t n4, const float* __restrict__ at,
                                                   const float* __restrict__ bt, int tail, double* partial) {
  pdl_enter();
  double S = 0.0;
  float C = 0.0f;
  const int64_t stride = int64_t(kDotBlocks) * 256;
  int64_t i = blockIdx.x * int64_t(256) + threadIdx.x;
  // four strides' loads in flight before their (in-order) accumulation
  for (; i + 3 * stride < n4; i += 4 * stride) {
    const float4 x0 = a[i], y0 = b[i], x1 = a[i + stride], y1 = b[i + stride];
    const float4 x2 = a[i + 2 * stride], y2 = b[i + 2 * stride], x3 = a[i + 3 * stride], y3 = b[i + 3 * stride];
    dot4_exact(x0, y0, S, C);
    dot4_exact(x1, y1, S, C);
    dot4_exact(x2, y2, S, C);
    dot4_exact(x3, y3, S, C);
  }
  for (; i < n4; i += stride) dot4_exact(a[i], b[i], S, C);
  double s = __dadd_rn(S, double(C));
  if (blockIdx.x == 0 && threadIdx.x < tail) s = fma(double(at[threadIdx.x]), double(bt[threadIdx.x]), s);
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
cudaError_t launch_dot_partial(const T* a, const T* b, int64_t n, double* partial, cudaStream_t st) {
  ProfScope ps(KK_DOT, st, double(sizeof(T)) * n * 2, double(n) * 2);
  const bool aligned = (reinterpret_cast<uintptr_t>(a) % 16 == 0) && (reinterpret_cast<uintptr_t>(b) % 16 == 0);
  if (sizeof(T) == 4 && aligned) {
    const float* af = reinterpret_cast<const float*>(a);
    const float* bf = reinterpret_cast<const float*>(b);
    const int64_t n4 = n / 4;
    {
      const cudaError_t le_ = launch_pdl(dot4_kernel, dim3(kDotBlocks), dim3(256), size_t(0), st,
                                        reinterpret_cast<const float4*>(af), reinterpret_cast<const float4*>(bf), n4, af + 4 * n4, bf + 4 * n4, int(n - 4 * n4), partial);
      if (le_ != cudaSuccess) return le_;
    }
  } else {
    {
      const cudaError_t le_ = launch_pdl(dot_kernel<T>, dim3(kDotBlocks), dim3(256), size_t(0), st,
                                        a, b, n, partial);
      if (le_ != cudaSuccess) return le_;
    }
  }
  note_launch();
  return cudaGetLastError();
}

__device__ double reduce_partials(const double* partial) {
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += 256) s += partial[i];
  return block_sum<256>(s);
}

__global__ void sum_partials_kernel(const double* partial, double* out) {
  pdl_enter();
  const double s = reduce_partials(partial);
  if (threadIdx.x == 0) *out = s;
}

cudaError_t launch_sum_partials(const double* partial, double* out, cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 8.0 * kDotBlocks, 2.0 * kDotBlocks);
  {
    const cudaError_t le_ = launch_pdl(sum_partials_kernel, dim3(1), dim3(256), size_t(0), st,
                                      partial, out);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

__global__ void minres_init_kernel(MinresState* s, const double* partial, double target) {
  pdl_enter();
  const double vz = reduce_partials(partial);
  if (threadIdx.x != 0) return;
  s->dot = vz;
  s->flag = 0;
  s->iter = 0;
  s->wx_pending = 0;
  s->w_q = s->w_m1 = s->w_m2 = s->x_w = 0.0;
  if (!(vz > 0.0)) { s->flag = (vz == vz) ? 3 : 4; s->beta = 1.0; s->beta1 = 1.0; s->est = 1.0; return; }
  s->beta = sqrt(vz);
  s->beta1 = s->beta;
  s->beta_prev = 1.0;
  s->eta = s->beta;
  s->c_m1 = s->c_m2 = 1.0;
  s->s_m1 = s->s_m2 = 0.0;
  s->est = 1.0;
  s->target = target;
}

__global__ void minres_alpha_kernel(MinresState* s, const double* partial) {
  pdl_enter();
  const double zkz = reduce_partials(partial);
  if (threadIdx.x != 0) return;
  const double b = s->beta;
  s->dot = zkz;
  s->alpha = zkz / (b * b);                 // q^T K q with q = z / beta
  s->coef_q = 1.0 / b;
  s->coef_v = s->alpha / b;
  s->coef_vp = s->iter == 0 ? 0.0 : b / s->beta_prev;
  if (!(s->alpha == s->alpha)) s->flag = 4;
}

__global__ void minres_rotate_kernel(MinresState* s, const double* partial) {
  pdl_enter();
  const double vz = reduce_partials(partial);
  if (threadIdx.x != 0) return;
  s->dot = vz;
  s->wx_pending = 0;
  if (!(vz == vz)) { s->flag = 4; return; }
  if (vz < 0.0) { s->flag = 3; return; }
  const double bn = sqrt(vz);
  const double b = s->beta, al = s->alpha;
  const double eps = s->s_m2 * b;
  const double dprime = s->c_m2 * b;
  const double delta = s->c_m1 * dprime + s->s_m1 * al;
  const double gbar = -s->s_m1 * dprime + s->c_m1 * al;
  const double rho = hypot(gbar, bn);
  if (rho == 0.0) { s->flag = 2; s->w_q = s->w_m1 = s->w_m2 = s->x_w = 0.0; return; }
  const double c = gbar / rho, sn = bn / rho;
  s->eps = eps; s->delta = delta; s->rho = rho; s->c = c; s->s = sn;
  s->w_q = 1.0 / (b * rho);
  s->w_m1 = delta / rho;
  s->w_m2 = eps / rho;
  s->x_w = c * s->eta;
  s->eta = -sn * s->eta;
  s->est = fabs(s->eta) / s->beta1;
  s->c_m2 = s->c_m1; s->s_m2 = s->s_m1;
  s->c_m1 = c; s->s_m1 = sn;
  s->beta_prev = b;
  s->beta = bn;
  s->iter += 1;
  s->wx_pending = 1;
  if (!(s->est == s->est)) s->flag = 4;
  else if (s->est <= s->target) s->flag = 1;
  else if (bn == 0.0) s->flag = 2;
}

cudaError_t launch_minres_init(MinresState* s, const double* partial, double target, cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 8.0 * kDotBlocks, 2.0 * kDotBlocks);
  {
    const cudaError_t le_ = launch_pdl(minres_init_kernel, dim3(1), dim3(256), size_t(0), st,
                                      s, partial, target);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_minres_alpha(MinresState* s, const double* partial, cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 8.0 * kDotBlocks, 2.0 * kDotBlocks);
  {
    const cudaError_t le_ = launch_pdl(minres_alpha_kernel, dim3(1), dim3(256), size_t(0), st,
                                      s, partial);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_minres_rotate(MinresState* s, const double* partial, cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 8.0 * kDotBlocks, 2.0 * kDotBlocks);
  {
    const cudaError_t le_ = launch_pdl(minres_rotate_kernel, dim3(1), dim3(256), size_t(0), st,
                                      s, partial);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void minres_v_kernel(const T* __restrict__ Kz, const T* __restrict__ v, T* vprev, int64_t n,
                                const MinresState* s) {
  pdl_enter();
  const T cq = T(s->coef_q), cv = T(s->coef_v), cvp = T(s->coef_vp);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    T r = cq * Kz[i] - cv * v[i];
    if (cvp != T(0)) r -= cvp * vprev[i];
    vprev[i] = r;
  }
}

template <typename T, typename TX>
__global__ void minres_wx_kernel(const T* __restrict__ z, const T* __restrict__ wm1, T* wm2, TX* x, int64_t n,
                                 const MinresState* s) {
  pdl_enter();
  const T wq = T(s->w_q), w1 = T(s->w_m1), w2 = T(s->w_m2);
  const TX xw = TX(s->x_w);
  if (!s->wx_pending) return;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const T w = wq * z[i] - w1 * wm1[i] - w2 * wm2[i];
    wm2[i] = w;
    x[i] += xw * TX(w);
  }
}

// float32 forms of the two updates on float4 packets; the n % 4 tail entries
// are done by the first threads of block 0
__global__ void minres_v4_kernel(const float4* __restrict__ Kz, const float4* __restrict__ v, float4* vprev,
                                 int64_t n4, const float* Kzt, const float* vt, float* vpt, int tail,
                                 const MinresState* s) {
  pdl_enter();
  const float cq = float(s->coef_q), cv = float(s->coef_v), cvp = float(s->coef_vp);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
    const float4 k = Kz[i], a = v[i];
    float4 r = make_float4(cq * k.x - cv * a.x, cq * k.y - cv * a.y, cq * k.z - cv * a.z, cq * k.w - cv * a.w);
    if (cvp != 0.f) {
      const float4 p = vprev[i];
      r.x -= cvp * p.x; r.y -= cvp * p.y; r.z -= cvp * p.z; r.w -= cvp * p.w;
    }
    vprev[i] = r;
  }
  if (blockIdx.x == 0 && threadIdx.x < tail) {
    const int i = threadIdx.x;
    float r = cq * Kzt[i] - cv * vt[i];
    if (cvp != 0.f) r -= cvp * vpt[i];
    vpt[i] = r;
  }
}

__global__ void minres_wx4_kernel(const float4* __restrict__ z, const float4* __restrict__ wm1, float4* wm2,
                                  float4* x, int64_t n4, const float* zt, const float* w1t, float* w2t, float* xt,
                                  int tail, const MinresState* s) {
  pdl_enter();
  const float wq = float(s->w_q), w1 = float(s->w_m1), w2 = float(s->w_m2), xw = float(s->x_w);
  if (!s->wx_pending) return;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
    const float4 a = z[i], b = wm1[i], c = wm2[i];
    float4 xv = x[i];
    const float4 w = make_float4(wq * a.x - w1 * b.x - w2 * c.x, wq * a.y - w1 * b.y - w2 * c.y,
                                 wq * a.z - w1 * b.z - w2 * c.z, wq * a.w - w1 * b.w - w2 * c.w);
    wm2[i] = w;
    xv.x += xw * w.x; xv.y += xw * w.y; xv.z += xw * w.z; xv.w += xw * w.w;
    x[i] = xv;
  }
  if (blockIdx.x == 0 && threadIdx.x < tail) {
    const int i = threadIdx.x;
    const float w = wq * zt[i] - w1 * w1t[i] - w2 * w2t[i];
    w2t[i] = w;
    xt[i] += xw * w;
  }
}

static bool al16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

template <typename T>
cudaError_t launch_minres_v(const T* Kz, const T* v, T* vprev, int64_t n, const MinresState* s, cudaStream_t st) {
  ProfScope ps(KK_VECTOR, st, double(sizeof(T)) * n * 4, double(n) * 5);
  if (sizeof(T) == 4 && al16(Kz) && al16(v) && al16(vprev)) {
    const float* k = reinterpret_cast<const float*>(Kz);
    const float* a = reinterpret_cast<const float*>(v);
    float* p = reinterpret_cast<float*>(vprev);
    const int64_t n4 = n / 4;
    {
      const cudaError_t le_ = launch_pdl(minres_v4_kernel, dim3(grid_for(n4, 256)), dim3(256), size_t(0), st,
                                         reinterpret_cast<const float4*>(k), reinterpret_cast<const float4*>(a), reinterpret_cast<float4*>(p), n4, k + 4 * n4, a + 4 * n4, p + 4 * n4, int(n - 4 * n4), s);
      if (le_ != cudaSuccess) return le_;
    }
  } else {
    {
      const cudaError_t le_ = launch_pdl(minres_v_kernel<T>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                        Kz, v, vprev, n, s);
      if (le_ != cudaSuccess) return le_;
    }
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t launch_minres_wx(const T* z, const T* wm1, T* wm2, TX* x, int64_t n, const MinresState* s,
                             cudaStream_t st) {
  ProfScope ps(KK_VECTOR, st, double(sizeof(T)) * n * 4 + double(sizeof(TX)) * n * 2, double(n) * 8);
  if (sizeof(T) == 4 && sizeof(TX) == 4 && al16(z) && al16(wm1) && al16(wm2) && al16(x)) {
    const float* a = reinterpret_cast<const float*>(z);
    const float* b = reinterpret_cast<const float*>(wm1);
    float* c = reinterpret_cast<float*>(wm2);
    float* xf = reinterpret_cast<float*>(x);
    const int64_t n4 = n / 4;
    {
      const cudaError_t le_ = launch_pdl(minres_wx4_kernel, dim3(grid_for(n4, 256)), dim3(256), size_t(0), st,
                                         reinterpret_cast<const float4*>(a), reinterpret_cast<const float4*>(b), reinterpret_cast<float4*>(c), reinterpret_cast<float4*>(xf), n4, a + 4 * n4, b + 4 * n4, c + 4 * n4, xf + 4 * n4, int(n - 4 * n4), s);
      if (le_ != cudaSuccess) return le_;
    }
  } else {
    {
      const cudaError_t le_ = launch_pdl(minres_wx_kernel<T, TX>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                        z, wm1, wm2, x, n, s);
      if (le_ != cudaSuccess) return le_;
    }
  }
  note_launch();
  return cudaGetLastError();
}

template <typename TA, typename TB>
__global__ void convert_kernel(const TA* a, TB* b, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = TB(a[i]);
}
template <typename TA, typename TB>
cudaError_t launch_convert(const TA* a, TB* b, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, double(sizeof(TA) + sizeof(TB)) * n, 0.0);
  {
    const cudaError_t le_ = launch_pdl(convert_kernel<TA, TB>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                      a, b, n);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

__global__ void sub_kernel(const double* a, const double* b, double* y, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = a[i] - b[i];
}
cudaError_t launch_sub(const double* a, const double* b, double* y, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, 24.0 * n, 0.0);
  {
    const cudaError_t le_ = launch_pdl(sub_kernel, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                      a, b, y, n);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void add_to_kernel(const T* d, double* x, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] += double(d[i]);
}
template <typename T>
cudaError_t launch_add_to(const T* d, double* x, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, (sizeof(T) + 16.0) * n, 0.0);
  {
    const cudaError_t le_ = launch_pdl(add_to_kernel<T>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                      d, x, n);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

__global__ void add_scaled_kernel(const float* d, double* x, int64_t n, double a) {
  pdl_enter();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = fma(a, double(d[i]), x[i]);
}
cudaError_t launch_add_scaled(const float* d, double* x, int64_t n, double a, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, 20.0 * n, 0.0);
  {
    const cudaError_t le_ = launch_pdl(add_scaled_kernel, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                      d, x, n, a);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

__global__ void scale_to32_kernel(const double* x, float* y, int64_t n, double a) {
  pdl_enter();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = float(a * x[i]);
}
cudaError_t launch_scale_to32(const double* x, float* y, int64_t n, double a, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, 12.0 * n, 0.0);
  {
    const cudaError_t le_ = launch_pdl(scale_to32_kernel, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                      x, y, n, a);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void fill_kernel(T* x, int64_t n, T v) {
  pdl_enter();
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) x[i] = v;
}
template <typename T>
cudaError_t launch_fill(T* x, int64_t n, T v, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ProfScope ps(KK_VECTOR, st, double(sizeof(T)) * n, 0.0);
  {
    const cudaError_t le_ = launch_pdl(fill_kernel<T>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st,
                                      x, n, v);
    if (le_ != cudaSuccess) return le_;
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FGMRES kernels (Arnoldi with classical Gram-Schmidt and one reorthogonalisation:
// each pass is one multi-dot and one multi-axpy over all basis vectors instead of
// j + 1 dependent dot/axpy pairs).  Inner products in float64 (float32 operands by
// the error-free float32 transformations of dot4_kernel); vector updates in the
// vectors' type with the float64 coefficients rounded to it.
// ---------------------------------------------------------------------------
// one basis vector's partial inner product over a block's chunk: float64 operands in
// float64; float32 operands four at a time by the error-free transformations of dot4_kernel
// (V_i and w 16-byte aligned: ldv and the chunk are multiples of four entries)
template <typename T>
__device__ __forceinline__ double fg_partial(const T* __restrict__ v, const T* __restrict__ w, int64_t i0, int64_t i1);
template <>
__device__ __forceinline__ double fg_partial<double>(const double* __restrict__ v, const double* __restrict__ w,
                                                    int64_t i0, int64_t i1) {
  double S = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) S = fma(v[i], w[i], S);
  return S;
}
template <>
__device__ __forceinline__ double fg_partial<float>(const float* __restrict__ v, const float* __restrict__ w,
                                                   int64_t i0, int64_t i1) {
  double S = 0.0;
  float C = 0.0f;
  const int64_t q0 = i0 >> 2, q1 = i1 >> 2;            // whole float4 groups of the chunk
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const float4* w4 = reinterpret_cast<const float4*>(w);
  for (int64_t q = q0 + threadIdx.x; q < q1; q += 256) dot4_exact(v4[q], w4[q], S, C);
  double r = __dadd_rn(S, double(C));
  for (int64_t i = (q1 << 2) + threadIdx.x; i < i1; i += 256) r = fma(double(v[i]), double(w[i]), r);
  return r;
}

template <typename T>
__global__ void __launch_bounds__(256) fgmres_multidot_kernel(const T* __restrict__ V, int64_t ldv,
                                                              const T* __restrict__ w, int64_t n,
                                                              const FgmresState* s, double* partial) {
  pdl_enter();
  const int count = s->j + 1;
  const int64_t chunk = ((n + kDotBlocks - 1) / kDotBlocks + 3) & ~int64_t(3);
  const int64_t i0 = min(n, int64_t(blockIdx.x) * chunk), i1 = min(n, i0 + chunk);
  for (int c = 0; c < count; ++c) {
    const double r = block_sum<256>(fg_partial<T>(V + int64_t(c) * ldv, w, i0, i1));
    if (threadIdx.x == 0) partial[int64_t(c) * kDotBlocks + blockIdx.x] = r;
  }
}

__global__ void fgmres_reduce_kernel(FgmresState* s, const double* partial, int second) {
  pdl_enter();
  const int c = blockIdx.x;
  if (c > s->j) return;
  const double r = reduce_partials(partial + int64_t(c) * kDotBlocks);
  if (threadIdx.x == 0) (second ? s->h2 : s->h)[c] = r;
}

template <typename T>
cudaError_t launch_fgmres_multidot(const T* V, int64_t ldv, const T* w, int64_t n, FgmresState* s, int second,
                                   double* partial, cudaStream_t st) {
  ProfScope ps(KK_DOT, st, double(sizeof(T)) * n * 2, double(n) * 2);
  cudaError_t e = launch_pdl(fgmres_multidot_kernel<T>, dim3(kDotBlocks), dim3(256), size_t(0), st, V, ldv, w, n,
                             static_cast<const FgmresState*>(s), partial);
  if (e != cudaSuccess) return e;
  note_launch();
  e = launch_pdl(fgmres_reduce_kernel, dim3(kFgmresMax + 1), dim3(256), size_t(0), st, s,
                 static_cast<const double*>(partial), second);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// mode 0: w -= sum_{c <= j} h[c] V_c; mode 1: the same with h2; mode 2: w += sum_{c < j} y[c] V_c
template <typename T, typename TX>
__global__ void __launch_bounds__(256) fgmres_axpy_kernel(TX* w, const T* __restrict__ V, int64_t ldv, int64_t n,
                                                          const FgmresState* s, int mode) {
  pdl_enter();
  const int count = mode == 2 ? s->j : s->j + 1;
  const double* coef = mode == 0 ? s->h : mode == 1 ? s->h2 : s->y;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    TX acc = w[i];
    for (int c = 0; c < count; ++c) {
      const TX cf = TX(coef[c]);
      acc = mode == 2 ? fma(cf, TX(V[int64_t(c) * ldv + i]), acc) : fma(-cf, TX(V[int64_t(c) * ldv + i]), acc);
    }
    w[i] = acc;
  }
}

template <typename T, typename TX>
cudaError_t launch_fgmres_axpy(TX* w, const T* V, int64_t ldv, int64_t n, const FgmresState* s, int mode,
                               cudaStream_t st) {
  ProfScope ps(KK_VECTOR, st, double(sizeof(T)) * n * 3, double(n) * 2);
  const cudaError_t e = launch_pdl(fgmres_axpy_kernel<T, TX>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st, w, V,
                                   ldv, n, s, mode);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

__global__ void fgmres_start_kernel(FgmresState* s, const double* partial, double target, double bnorm) {
  pdl_enter();
  const double rr = reduce_partials(partial);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(rr);
  s->beta = beta;
  s->target = target;
  s->bnorm = bnorm;
  s->est = beta / bnorm;
  s->j = 0;
  s->flag = (beta == beta) ? 0 : 4;
  s->g[0] = beta;
}

cudaError_t launch_fgmres_start(FgmresState* s, const double* partial, double target, double bnorm,
                                cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 8.0 * kDotBlocks, 2.0 * kDotBlocks);
  const cudaError_t e = launch_pdl(fgmres_start_kernel, dim3(1), dim3(256), size_t(0), st, s, partial, target, bnorm);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

__global__ void fgmres_rotate_kernel(FgmresState* s, const double* partial) {
  pdl_enter();
  const double ww = reduce_partials(partial);
  if (threadIdx.x != 0) return;
  const int j = s->j;
  constexpr int ld = kFgmresMax + 1;
  double* col = s->H + int64_t(j) * ld;
  for (int i = 0; i <= j; ++i) col[i] = s->h[i] + s->h2[i];
  const double hn = sqrt(ww);
  s->hnext = hn;
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {                        // previous rotations
    const double a = col[i], b = col[i + 1];
    col[i] = s->cs[i] * a + s->sn[i] * b;
    col[i + 1] = -s->sn[i] * a + s->cs[i] * b;
  }
  const double rho = hypot(col[j], col[j + 1]);
  s->j = j + 1;
  if (!(rho == rho) || !(hn == hn)) { s->flag = 4; return; }
  if (rho == 0.0) { s->flag = 2; return; }
  const double c = col[j] / rho, sn = col[j + 1] / rho;
  s->cs[j] = c; s->sn[j] = sn;
  col[j] = rho;
  col[j + 1] = 0.0;
  const double gj = s->g[j];
  s->g[j + 1] = -sn * gj;
  s->g[j] = c * gj;
  s->est = fabs(s->g[j + 1]) / s->bnorm;
  if (s->est <= s->target) s->flag = 1;
  else if (hn == 0.0) s->flag = 2;                    // lucky breakdown: the Krylov space is invariant
}

cudaError_t launch_fgmres_rotate(FgmresState* s, const double* partial, cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 8.0 * kDotBlocks, 2.0 * kDotBlocks);
  const cudaError_t e = launch_pdl(fgmres_rotate_kernel, dim3(1), dim3(256), size_t(0), st, s, partial);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

__global__ void fgmres_solve_y_kernel(FgmresState* s) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  const int k = s->j;
  constexpr int ld = kFgmresMax + 1;
  for (int i = k - 1; i >= 0; --i) {                   // back substitution with the rotated H
    double r = s->g[i];
    for (int c = i + 1; c < k; ++c) r -= s->H[int64_t(c) * ld + i] * s->y[c];
    s->y[i] = r / s->H[int64_t(i) * ld + i];
  }
}

cudaError_t launch_fgmres_solve_y(FgmresState* s, cudaStream_t st) {
  ProfScope ps(KK_SCALAR, st, 0.0, 0.0);
  const cudaError_t e = launch_pdl(fgmres_solve_y_kernel, dim3(1), dim3(32), size_t(0), st, s);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void fgmres_scale_kernel(const T* __restrict__ in, T* out, int64_t n, const FgmresState* s, int which) {
  pdl_enter();
  const double d = which == 0 ? s->beta : s->hnext;
  const T a = T(d != 0.0 ? 1.0 / d : 0.0);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = a * in[i];
}

template <typename T>
cudaError_t launch_fgmres_scale(const T* in, T* out, int64_t n, const FgmresState* s, int which, cudaStream_t st) {
  ProfScope ps(KK_VECTOR, st, double(sizeof(T)) * n * 2, double(n));
  const cudaError_t e = launch_pdl(fgmres_scale_kernel<T>, dim3(grid_for(n, 256)), dim3(256), size_t(0), st, in, out,
                                   n, s, which);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

// explicit instantiations
#define SGOC_INST(T)                                                                                               \
  template cudaError_t launch_sg<T>(const SGArgs<T>&, cudaStream_t);                                               \
  template cudaError_t launch_sg_variant<T>(const SGArgs<T>&, int, cudaStream_t, const SGMulti<T>*);            \
  template cudaError_t launch_sg_group<T>(const SGArgs<T>*, int, cudaStream_t);                                    \
  template int sg_tuned_variant<T>(const SGArgs<T>&);                                                              \
  template void sg_set_variant<T>(const SGArgs<T>&, int);                                                          \
  template void sg_clear_variant<T>(const SGArgs<T>&);                                                             \
  template bool sg_variant_feasible<T>(const SGArgs<T>&, int);                                                     \
  template cudaError_t launch_mass<T>(const MassArgs<T>&, cudaStream_t);                                           \
  template cudaError_t launch_cheb<T>(const ChebArgs<T>&, cudaStream_t);                                           \
  template cudaError_t launch_mass_exact<T>(const ChebArgs<T>&, const T*, const T*, cudaStream_t);                 \
  template cudaError_t launch_smooth<T>(const T*, const T*, T*, int64_t, int, Stencil, T, T*, int64_t, int, int,   \
                                        cudaStream_t);                                                             \
  template cudaError_t launch_residual<T>(const T*, const T*, T*, int64_t, int, Stencil, cudaStream_t);            \
  template cudaError_t launch_restrict<T>(const T*, T*, int64_t, int, cudaStream_t);                               \
  template cudaError_t launch_prolong_add<T>(const T*, T*, int64_t, int, cudaStream_t);                            \
  template cudaError_t launch_scale<T>(const T*, T*, int64_t, T, cudaStream_t);                                    \
  template cudaError_t launch_vcycle_full<T>(const T*, T*, int64_t, const FusedLevels&, T, int, T*, int64_t, int,  \
                                             int, cudaStream_t, VColumns);                                                   \
  template cudaError_t launch_vcycle_full_group<T>(const T* const*, T* const*, T* const*, const FusedLevels*, int,  \
                                                   int64_t, T, int, int64_t, int, int, cudaStream_t, VColumns);    \
  template cudaError_t launch_vcycle_cluster<T>(const T*, T*, int64_t, const ClusterLevels&, int, T, int, T*,      \
                                                int64_t, int, int, cudaStream_t);                                  \
  template cudaError_t launch_dot_partial<T>(const T*, const T*, int64_t, double*, cudaStream_t);                  \
  template cudaError_t launch_minres_v<T>(const T*, const T*, T*, int64_t, const MinresState*, cudaStream_t);      \
  template cudaError_t launch_add_to<T>(const T*, double*, int64_t, cudaStream_t);                                 \
  template cudaError_t launch_fill<T>(T*, int64_t, T, cudaStream_t);

SGOC_INST(float)
SGOC_INST(double)
template cudaError_t launch_fgmres_multidot<float>(const float*, int64_t, const float*, int64_t, FgmresState*, int,
                                                   double*, cudaStream_t);
template cudaError_t launch_fgmres_multidot<double>(const double*, int64_t, const double*, int64_t, FgmresState*,
                                                    int, double*, cudaStream_t);
template cudaError_t launch_fgmres_axpy<float, float>(float*, const float*, int64_t, int64_t, const FgmresState*,
                                                      int, cudaStream_t);
template cudaError_t launch_fgmres_axpy<double, double>(double*, const double*, int64_t, int64_t,
                                                        const FgmresState*, int, cudaStream_t);
template cudaError_t launch_fgmres_scale<float>(const float*, float*, int64_t, const FgmresState*, int, cudaStream_t);
template cudaError_t launch_fgmres_scale<double>(const double*, double*, int64_t, const FgmresState*, int,
                                                 cudaStream_t);
template cudaError_t launch_minres_wx<double, double>(const double*, const double*, double*, double*, int64_t,
                                                      const MinresState*, cudaStream_t);
template cudaError_t launch_minres_wx<float, float>(const float*, const float*, float*, float*, int64_t,
                                                    const MinresState*, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);

}  // namespace sgoc
