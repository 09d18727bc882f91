// Exact mean solves by fast diagonalisation, on the tensor cores (tcgen05).
//
// Every mean solve of the preconditioner is a solve with a constant 9-point stencil
// (d, e, c) of Q1 elements on a uniform grid with homogeneous Dirichlet boundary: the
// steady A~_1 = kappa0 K + s M (Eq. (mathcalZ)) and the time slab operator
// A^_1 = (1 + tau s) M + tau kappa0 K (Eq. (A_hat)).  In tensor form both 1-D factors
// are tridiagonal Toeplitz matrices, diagonalised by the orthonormal type-I sine
// transform S, S_pi = sqrt(2/(n1+1)) sin(pi (p+1)(i+1)/(n1+1)) (symmetric, S S = I):
//   A = (S (x) S) Lambda (S (x) S),
//   lambda_ij = d + 2e (cos th_i + cos th_j) + 4c cos th_i cos th_j,  th_i = pi (i+1)/(n1+1).
// With a column of the batch as the n1 x n1 matrix X (rows y, columns x),
//   A^{-1} X = S (Lambda^{-1} o (S X S)) S,
// four dense products with the constant S: the exact B = A~_1^{-1} of Alg. 1 (the
// paper's hierarchical Gauss-Seidel) in place of one V-cycle.
//
// Layout on the tensor cores.  A tile holds 128 / NB columns of NB = n1 + 1 (padded) rows
// stacked along M = 128; each product is D = A B with A (M x K) in tensor memory (row m on
// lane m), B (K x N) in shared memory and D (128 lanes x NB columns, float32) in tensor memory:
//   G1  D1 = X S          A = X,                    B = S_NB (K-major)
//   G2  D2 = S D1         A = S_128,                B = D1   (MN-major)
//   --  Yh = Lambda^{-1} o D2 (per element, in registers)
//   G3  D3 = Yh S         A = Yh,                   B = S_NB (K-major)
//   G4  D4 = S D3         A = S_128,                B = D3   (MN-major)
// S_128 is block-diagonal with 128 / NB copies of S_NB; it is put into tensor memory once per
// CTA.  Thread r of the 128 owns row r (tensor-memory lane r) of every D and writes its row of
// the next operand: into its own lane when that operand is an A, as K row r of the MN-major B
// of G2 / G4 otherwise, so no transpose is needed.  The shared-memory operands use the
// 128-byte swizzled canonical layouts.
//
// Precision.  Both factors of every product are split into two bfloat16 terms
// (v = hi + lo, hi = bf16(v), lo = bf16(v - hi)); a product accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi in float32, so it carries about 16 bits of both
// operands (relative error ~2^-16, against 2^-24 for float32 arithmetic and ~0.1 for the
// V-cycle's contraction): the operator applied is the exact inverse to about 1e-5.
#include "kernels.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

namespace sgoc {

namespace {

constexpr int kSpecThreads = 512;        // four warps per tensor-memory lane quarter
// tensor-memory columns: the float32 accumulator (0 ..), the table of 1 / lambda (128 ..), the
// split transform S_128 as the A operand of the left products (hi 256 .., lo 320 ..) and the
// split data as the A operand of the right products (hi 384 .., lo 448 ..)
constexpr uint32_t kSpecTmemCols = 512;
constexpr uint32_t kColTab = 128, kColSh = 256, kColSl = 320, kColXh = 384, kColXl = 448;
static_assert(kColTab >= 128 && kColSh >= kColTab + 128 && kColSl >= kColSh + 64 && kColXh >= kColSl + 64 &&
                  kColXl >= kColXh + 64 && kColXl + 64 <= kSpecTmemCols,
              "accumulator (NB columns), table (NB), S_128 hi / lo (64 each), data hi / lo (NB / 2 each)");
constexpr int kSpecSpin = 1 << 20;       // bounded mbarrier polls before the kernel gives up

template <int NB>
struct SpecGeo {
  static_assert(NB == 64 || NB == 128, "padded grid sizes 64 and 128");
  static constexpr int CPT = 128 / NB;                 // grid columns per tile
  static constexpr int N1 = NB - 1;                    // interior nodes per side
  static constexpr int N0 = N1 * N1;
  static constexpr int KSTEPS_NB = NB / 16;            // bf16 MMA steps (K = 16) over NB
  static constexpr int SA = 128 * 128 * 2;             // one bf16 128 x 128 operand
  static constexpr int SB = NB == 128 ? 0 : NB * NB * 2;
  static constexpr int DAT = 128 * NB * 2;             // one bf16 data operand
  static constexpr int oSAh = 0, oSAl = SA;
  static constexpr int oSBh = NB == 128 ? oSAh : 2 * SA;
  static constexpr int oSBl = NB == 128 ? oSAl : 2 * SA + SB;
  static constexpr int oT = 2 * SA + 2 * SB;           // mode table t_i = 1 - cos th_i
  static constexpr int IMG = oT + NB * 4;              // bytes of the constant image
  static constexpr int oDh = (IMG + 1023) / 1024 * 1024;
  static constexpr int oDl = oDh + DAT;
  static constexpr int STG = (N0 * 4 + 16 + 15) / 16 * 16;   // float32 column in its global layout
  static constexpr int oStg = oDl + DAT;               // CPT staging columns (input, then output)
  static constexpr int oBar = oStg + CPT * STG;        // three mbarriers
  static constexpr int oTm = oBar + 24;                // tensor-memory address
  static constexpr int SMEM = oTm + 16 + 1024;         // + slack to align the base to 1024
  static constexpr int SBO_MN = (NB / 64) * 1024;      // MN-major: stride of 8-row K groups
};

static_assert(SpecGeo<128>::SMEM <= 232448 && SpecGeo<64>::SMEM <= 232448, "shared memory of one CTA");
static_assert(SpecGeo<128>::oBar % 8 == 0 && SpecGeo<64>::oBar % 8 == 0, "mbarriers are 8-byte aligned");

// byte offset of element (r, k) of an R-row, K-major operand, 128-byte swizzle:
// 8-row x 128-byte atoms, 16-byte chunks XOR-ed with the row within the atom,
// atoms along K (64 bf16) at R / 8 * 1024 bytes
__host__ __device__ constexpr int off_kmajor(int R, int r, int k) {
  return (k >> 6) * (R / 8 * 1024) + (r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) & 7) ^ (r & 7)) << 4) +
         (k & 7) * 2;
}
// byte offset of element (k, n) of a K x N MN-major operand, 128-byte swizzle: rows are
// K indices, 64 n per 128-byte atom row, atoms along N at 1024 bytes, 8-row K groups at sbo
__host__ __device__ constexpr int off_mnmajor(int sbo, int k, int n) {
  return (k >> 3) * sbo + (n >> 6) * 1024 + (k & 7) * 128 + ((((n >> 3) & 7) ^ (k & 7)) << 4) + (n & 7) * 2;
}

// ------------------------------------------------------------ PTX wrappers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void spec_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void spec_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false when the polls ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kSpecSpin; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 1-D bulk copy global -> shared, completing `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// 1-D bulk copy shared -> global, and its float32 add-reduction form (bulk group completion)
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_s2g_add(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// A float32 column of n0 values at global address g, staged in shared memory at stage + (g & 15)
// + 4 i (stage 16-byte aligned): the 16-byte aligned middle [lo, hi) moves by bulk copy, the
// at most three values before lo (head) and after hi (tail) by ordinary accesses.
struct StageSpan {
  uint32_t off;      // g & 15: byte offset of value 0 in the staging column
  int i_lo, i_hi;    // values [i_lo, i_hi) form the aligned middle
};
__device__ __forceinline__ StageSpan stage_span(const void* g, int n0) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(g), a1 = a0 + uintptr_t(n0) * 4;
  const uintptr_t lo = (a0 + 15) & ~uintptr_t(15), hi = a1 & ~uintptr_t(15);
  StageSpan sp;
  sp.off = uint32_t(a0 & 15);
  sp.i_lo = int((lo - a0) / 4);
  sp.i_hi = hi > lo ? int((hi - a0) / 4) : sp.i_lo;
  return sp;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor, 128-byte swizzle (sm_100 format: version bit 46,
// layout type 2 in bits 61-63), start address, leading and stride byte offsets >> 4
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}
// instruction descriptor of kind::f16: float32 accumulator (bits 4-5 = 1), bf16 A and B
// (bits 7-9, 10-12 = 1), A K-major, B K-major or MN-major (bit 16), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(b_mn ? 1 : 0) << 16) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}
// D (+)= A B, one M = 128, K = 16 step issued by this thread: A in tensor memory (row m on lane
// m, two bf16 of consecutive K per 32-bit column, the lower K in the low half), B in shared
// memory by descriptor, D in tensor memory; the previous D is kept when acc != 0
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 consecutive float32 columns of this thread's lane; the wait is part of the same
// statement, so no use of the values can be scheduled before the load completes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]) {
  static_assert(N == 16 || N == 32, "16 or 32 columns");
  if constexpr (N == 32) tmem_ld32(taddr, v);
  else tmem_ld16(taddr, v);
}

// store N (8 or 16) 32-bit columns of this thread's lane, and wait for the store to complete
template <int N>
__device__ __forceinline__ void tmem_st_u32(uint32_t taddr, const uint32_t (&v)[N]) {
  static_assert(N == 8 || N == 16, "8 or 16 columns");
  if constexpr (N == 16) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};\n"
        "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
  } else {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
        "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
  }
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// v = hi + lo with hi = bf16(v), lo = bf16(v - hi), for a pair; packed bf16x2 words
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// D = A B over K = 16 * ksteps with the split operands, A_hi B_hi + A_hi B_lo + A_lo B_hi: A in
// tensor memory (k-step s at columns a_hi / a_lo + 8 s), B in shared memory (k-step s at byte
// offset b_step(s) of its region)
template <typename FB>
__device__ __forceinline__ void gemm_split_ts(uint32_t tmem_d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                              uint32_t b_lo, uint32_t b_lbo, uint32_t b_sbo, uint32_t idesc, int ksteps,
                                              FB b_step) {
  for (int s = 0; s < ksteps; ++s) {
    const uint32_t bo = b_step(s), ao = uint32_t(8 * s);
    const uint64_t bh = sw128_desc(b_hi + bo, b_lbo, b_sbo);
    tc_mma_ts(tmem_d, a_hi + ao, bh, idesc, s > 0 ? 1u : 0u);
    tc_mma_ts(tmem_d, a_hi + ao, sw128_desc(b_lo + bo, b_lbo, b_sbo), idesc, 1u);
    tc_mma_ts(tmem_d, a_lo + ao, bh, idesc, 1u);
  }
}

}  // namespace

// set when a bounded wait of the kernel ran out (the tensor cores or the bulk copy never
// signalled); read and cleared by spectral_take_error
__device__ int g_spec_err = 0;

// Exact mean solves of B columns.  Column col's right-hand side is read at
// b + (col / b_L) b_ss + (col % b_L) n0 when cols.b_L > 0, else at b + col n0; its solution
// goes to x + col n0, or with acc to acc + (col / acc_L) acc_ss + (acc_col0 + col % acc_L) n0,
// added when cols.acc_add (the V-cycle's conventions).  img is the constant image of the
// split S operands and the mode table; (l0, l1, l2) the eigenvalue coefficients,
// lambda_ij = l0 + l1 (t_i + t_j) + l2 t_i t_j with t_i = 1 - cos th_i.
// 512 threads: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its lane quarter) and
// takes the column quarter w / 4 of every accumulator row; thread 0 issues the products.
// PREC 0: both factors of every product split (hi*hi + hi*lo + lo*hi, the exact solve), the
// only form launched.  Measured and dropped: 1, the transform rounded to bfloat16 with the
// data split (two products; 2.7e-3 from the exact inverse at 128 x 128), and 2, both rounded
// (one product; also nonlinear at 5e-3).  The conditioning of the mean operator amplifies the
// transform's rounding through the hGS sweep: at beta = 1e-2 the mixed 128 x 128 solve took
// 351 (form 1) and 9000 (form 2) inner iterations instead of 43.
// Merged launches (several problems of one grid): member g's tiles are blocks
// [g * tiles, (g + 1) * tiles) of the grid, with its own right-hand sides, outputs and
// eigenvalue coefficients selected by constant indices (they stay in parameter space).
template <int NB, int PREC>
__global__ void __launch_bounds__(kSpecThreads, 1)
    spectral_mean_kernel(const float* __restrict__ bg, float* xg, int64_t B, const uint8_t* __restrict__ img,
                         float l0, float l1, float l2, float* acc, int64_t acc_ss, int acc_L, int acc_col0,
                         VColumns cols, const SpecMulti sm_, const SpecScale sc) {
  using G = SpecGeo<NB>;
  int64_t tile = blockIdx.x;
  if (sm_.ng > 1) {
    const int64_t tiles = (B + G::CPT - 1) / G::CPT;
    const int g = int(tile / tiles);
    tile -= int64_t(g) * tiles;
#pragma unroll
    for (int i = 1; i < kMaxGroup; ++i)
      if (i == g) {
        bg = sm_.b[i]; xg = sm_.x[i]; acc = sm_.acc[i]; l0 = sm_.l0[i]; l1 = sm_.l1[i]; l2 = sm_.l2[i];
      }
  }
  constexpr int NW = kSpecThreads / 32;              // warps
  constexpr int CPW = NB / (NW / 4);                 // accumulator columns per warp (16 or 32)
  extern __shared__ uint8_t spec_raw[];
  const uint32_t raw = smem_u32(spec_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  const uint8_t* sm = spec_raw + pad;
  const uint32_t s0 = raw + pad;                     // 1024-aligned: the swizzle atoms' base
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = (warp & 3) * 32 + lane;            // accumulator row (tensor-memory lane)
  const int jbase = (warp >> 2) * CPW;               // first accumulator column of this thread
  const uint32_t bar_ld = s0 + G::oBar, bar_mma = s0 + G::oBar + 8, bar_in = s0 + G::oBar + 16;
  if (tid == 0) {
    mbar_init(bar_ld, 1);
    mbar_init(bar_mma, 1);
    mbar_init(bar_in, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(s0 + G::oTm, kSpecTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<const volatile uint32_t*>(sm + G::oTm);
  if (tid == 0) {                                    // constant data: before the dependency wait
    mbar_expect_tx(bar_ld, uint32_t(G::IMG));
    bulk_g2s(s0, img, uint32_t(G::IMG), bar_ld);
  }
  const int64_t col0 = tile * G::CPT;
  const float* bcol[G::CPT];
#pragma unroll
  for (int c = 0; c < G::CPT; ++c) {
    const int64_t col = col0 + c;
    bcol[c] = col >= B ? nullptr
                       : (cols.b_L > 0 ? bg + (col / cols.b_L) * cols.b_ss + (col % cols.b_L) * int64_t(G::N0)
                                       : bg + col * int64_t(G::N0));
  }
  spec_pdl_wait();                                   // the right-hand sides and outputs are shared
  // the tile's right-hand sides into the staging columns: aligned middles by bulk copy, the
  // at most three values before and after them by threads 8c .. 8c + 7
  StageSpan span[G::CPT];
#pragma unroll
  for (int c = 0; c < G::CPT; ++c)
    span[c] = bcol[c] != nullptr ? stage_span(bcol[c], G::N0) : StageSpan{0u, 0, 0};
  if (tid == 0) {
    uint32_t tx = 0;
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) tx += uint32_t(span[c].i_hi - span[c].i_lo) * 4u;
    mbar_expect_tx(bar_in, tx);
#pragma unroll
    for (int c = 0; c < G::CPT; ++c)
      if (span[c].i_hi > span[c].i_lo)
        bulk_g2s(s0 + G::oStg + c * G::STG + span[c].off + 4u * span[c].i_lo, bcol[c] + span[c].i_lo,
                 uint32_t(span[c].i_hi - span[c].i_lo) * 4u, bar_in);
  }
#pragma unroll
  for (int c = 0; c < G::CPT; ++c) {
    const int j = tid - 8 * c;
    if (j >= 0 && j < 8 && bcol[c] != nullptr) {
      const int i = j < 4 ? j : span[c].i_hi + (j - 4);
      if (j < 4 ? i < span[c].i_lo : i < G::N0)
        *reinterpret_cast<float*>(spec_raw + pad + G::oStg + c * G::STG + span[c].off + 4 * i) = bcol[c][i];
    }
  }
  bool ok = mbar_wait(bar_ld, 0);
  // Constant data derived from the image, written into tensor memory while the tensor cores
  // work (after the image has landed): this thread's part of S_128, the A of the left products,
  // and the first half of its part of the table 1 / lambda_(mu, nu) (row mu = row mod NB,
  // columns jbase ..; tensor-memory columns kColTab + nu) during G1, the second half of the table
  // during G2 (the reciprocals are bound by the special-function units); the table is first read
  // by the scaling after G2.
  auto table = [&](int half) {
    const float* tt = reinterpret_cast<const float*>(sm + G::oT);
    const float tm = tt[row % NB];
    const float ar = fmaf(l1, tm, l0), br = fmaf(l2, tm, l1);
    // the column's scale factor (mass blocks), folded into the table
    float num = sc.mode == 2 ? sc.scale : 1.0f;
    if (sc.mode == 1) {
      const int64_t col = col0 + row / NB;
      const int64_t spc = int64_t(sc.slabs) * sc.P;
      const int64_t blk = col / spc, cc = col % spc;
      const int t = int(cc / sc.P), al = int(cc % sc.P);
      float sv = sc.nt > 0 ? sc.tau * ((sc.nt > 1 && (t == 0 || t == sc.nt - 1)) ? 0.5f : 1.0f) : 1.0f;
      sv *= blk == 0 ? (al == 0 ? 1.0f : 1.0f + sc.gamma) : sc.beta;
      num = 1.0f / sv;
    }
    constexpr int H = CPW / 2;
    const int j0 = jbase + half * H;
    uint32_t w[H];
#pragma unroll
    for (int i = 0; i < H; ++i) w[i] = __float_as_uint(__fdividef(num, fmaf(br, tt[j0 + i], ar)));
    tmem_st_u32<H>(tmem + (uint32_t((warp & 3) * 32) << 16) + kColTab + uint32_t(j0), w);
  };
  auto load_s = [&]() {
    // row `row` of the split S_128, K range 32 (warp / 4) .. (16-byte chunks of the K-major
    // image: 8 consecutive K each)
    const int kq = (warp >> 2) * 32;
    uint32_t sh[16], sl[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = off_kmajor(128, row, kq + 8 * i);
      const uint4 h = *reinterpret_cast<const uint4*>(sm + G::oSAh + o);
      const uint4 l = *reinterpret_cast<const uint4*>(sm + G::oSAl + o);
      sh[4 * i] = h.x; sh[4 * i + 1] = h.y; sh[4 * i + 2] = h.z; sh[4 * i + 3] = h.w;
      sl[4 * i] = l.x; sl[4 * i + 1] = l.y; sl[4 * i + 2] = l.z; sl[4 * i + 3] = l.w;
    }
    const uint32_t tq = tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t(kq / 2);
    tmem_st_u32<16>(tq + kColSh, sh);
    tmem_st_u32<16>(tq + kColSl, sl);

  };
  ok = mbar_wait(bar_in, 0) && ok;
  ok = __syncthreads_and(ok) != 0;
  const uint32_t trow = tmem + (uint32_t((warp & 3) * 32) << 16);   // this warp's lane quarter
  // v (this thread's accumulator columns jbase ..) split into the A operand of a right product:
  // row `row`, K = jbase .., two K per tensor-memory column
  auto store_a = [&](const float (&v)[CPW]) {
    uint32_t h[CPW / 2], l[CPW / 2];
#pragma unroll
    for (int i = 0; i < CPW / 2; ++i) split2(v[2 * i], v[2 * i + 1], h[i], l[i]);
    tmem_st_u32<CPW / 2>(trow + kColXh + uint32_t(jbase / 2), h);
    tmem_st_u32<CPW / 2>(trow + kColXl + uint32_t(jbase / 2), l);
  };
  // L: the staged right-hand sides as the A of G1: row r = c NB + y, K index x; the padding row
  // y = N1, column x = N1 and absent columns are zero.  Thread (row, jbase) reads x = jbase ..
  // of its row (the rows of a warp are N1 words apart: no bank conflicts).
  if (ok) {
    const int c = row / NB, y = row - c * NB;
    bool live = y < G::N1;
    uint32_t soff = 0;
#pragma unroll
    for (int i = 0; i < G::CPT; ++i)
      if (c == i) { live = live && bcol[i] != nullptr; soff = G::oStg + i * G::STG + span[i].off; }
    const float* sc = reinterpret_cast<const float*>(sm + soff) + y * G::N1;
    float v[CPW];
#pragma unroll
    for (int i = 0; i < CPW; ++i) v[i] = live && jbase + i < G::N1 ? sc[jbase + i] : 0.f;
    store_a(v);
  }
  tc_fence_before();

  constexpr uint32_t idK = idesc_bf16(128, NB, false), idMN = idesc_bf16(128, NB, true);
  const auto stepB = [](int s) { return uint32_t((s >> 2) * (NB / 8 * 1024) + (s & 3) * 32); }; // K-major, NB rows
  const auto stepMN = [](int s) { return uint32_t(s * 2 * G::SBO_MN); };                        // MN-major
  uint32_t parity = 0;
  // issue one product (thread 0) and wait for it (every thread)
  auto product = [&](bool left, auto&& during) {
    if (tid == 0) {
      tc_fence_after();
      // right products: A the data (tensor memory), B the transform S_NB (K-major); left
      // products: A the transform S_128 (tensor memory), B the data (MN-major)
      if (!left)
        gemm_split_ts(tmem, tmem + kColXh, tmem + kColXl, s0 + G::oSBh, s0 + G::oSBl, 16, 1024, idK, G::KSTEPS_NB,
                      stepB);
      else
        gemm_split_ts(tmem, tmem + kColSh, tmem + kColSl, s0 + G::oDh, s0 + G::oDl, 1024, G::SBO_MN, idMN, 8, stepMN);
      tc_commit(bar_mma);
    }
    __syncwarp();
    during();                                        // work that overlaps the product
    bool w = mbar_wait(bar_mma, parity);
    parity ^= 1u;
    w = __syncthreads_and(w) != 0;
    tc_fence_after();
    return w;
  };
  // this thread's part of accumulator row `row` -> split operand: the MN-major B of a left
  // product (K row `row`, shared memory), or, scaled by Lambda^{-1}, the A of a right product
  // (row `row`, tensor memory)
  auto store_row = [&](bool mn, bool scale) {
    float v[CPW];
    tmem_ld<CPW>(trow + uint32_t(jbase), v);
    if (scale) {
      float w[CPW];
      tmem_ld<CPW>(trow + kColTab + uint32_t(jbase), w);
#pragma unroll
      for (int i = 0; i < CPW; ++i) v[i] *= w[i];
    }
    if (mn) {
#pragma unroll
      for (int q = 0; q < CPW / 8; ++q) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split2(v[8 * q + 2 * i], v[8 * q + 2 * i + 1], h[i], l[i]);
        const int o = off_mnmajor(G::SBO_MN, row, jbase + 8 * q);
        sts128(s0 + G::oDh + o, h[0], h[1], h[2], h[3]);
        sts128(s0 + G::oDl + o, l[0], l[1], l[2], l[3]);
      }
      fence_async_smem();
    } else {
      store_a(v);
    }
    tc_fence_before();
    __syncthreads();
  };
  __syncthreads();
  const auto nothing = [] {};
  if (ok) ok = product(false, [&] { load_s(); table(0); });  // G1: D1 = X S
  if (ok) store_row(true, false);
  if (ok) ok = product(true, [&] { table(1); });     // G2: D2 = S D1 = S X S
  if (ok) store_row(false, true);                    // Lambda^{-1} o D2
  if (ok) ok = product(false, nothing);              // G3: D3 = Yh S
  if (ok) store_row(true, false);
  if (ok) ok = product(true, nothing);               // G4: D4 = S D3, the solution
  spec_pdl_trigger();                                // only the write of the solution remains
  if (ok) {
    // the solution rows into the staging columns in the global layout of each output column
    // (value i = y N1 + x at off + 4 i; rows of a warp are N1 words apart: no bank conflicts),
    // then bulk stores (or bulk float32 adds) of the aligned middles, the rest by threads
    const bool acc_on = acc != nullptr && cols.acc_add;
    float* gcol[G::CPT];
    StageSpan ospan[G::CPT];
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
      const int64_t col = col0 + c;
      gcol[c] = col >= B ? nullptr
                         : (acc != nullptr ? acc + (col / acc_L) * acc_ss + (acc_col0 + col % acc_L) * int64_t(G::N0)
                                           : xg + col * int64_t(G::N0));
      ospan[c] = gcol[c] != nullptr ? stage_span(gcol[c], G::N0) : StageSpan{0u, 0, 0};
    }
    {
      const int c = row / NB, y = row - c * NB;
      bool live = y < G::N1;
      uint32_t soff = 0;
#pragma unroll
      for (int i = 0; i < G::CPT; ++i)
        if (c == i) { live = live && gcol[i] != nullptr; soff = G::oStg + i * G::STG + ospan[i].off; }
      float* so = reinterpret_cast<float*>(spec_raw + pad + soff) + y * G::N1;
      float v[CPW];
      tmem_ld<CPW>(trow + uint32_t(jbase), v);
      if (live) {
#pragma unroll
        for (int i = 0; i < CPW; ++i)
          if (jbase + i < G::N1) so[jbase + i] = v[i];
      }
    }
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < G::CPT; ++c) {
        if (gcol[c] == nullptr || ospan[c].i_hi <= ospan[c].i_lo) continue;
        const uint32_t src = s0 + G::oStg + c * G::STG + ospan[c].off + 4u * ospan[c].i_lo;
        const uint32_t bytes = uint32_t(ospan[c].i_hi - ospan[c].i_lo) * 4u;
        if (acc_on) bulk_s2g_add(gcol[c] + ospan[c].i_lo, src, bytes);
        else bulk_s2g(gcol[c] + ospan[c].i_lo, src, bytes);
      }
      bulk_commit();
    }
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
      const int j = tid - 8 * c;
      if (j >= 0 && j < 8 && gcol[c] != nullptr) {
        const int i = j < 4 ? j : ospan[c].i_hi + (j - 4);
        if (j < 4 ? i < ospan[c].i_lo : i < G::N0) {
          const float v = *reinterpret_cast<const float*>(sm + G::oStg + c * G::STG + ospan[c].off + 4 * i);
          gcol[c][i] = acc_on ? gcol[c][i] + v : v;
        }
      }
    }
    if (tid == 0) bulk_wait_all();                   // the bulk writes are complete
  } else {
    if (tid == 0) atomicExch(&g_spec_err, 1);
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kSpecTmemCols);
  }
}

template <int NB>
std::vector<uint8_t> build_image(int n1) {
  using G = SpecGeo<NB>;
  std::vector<uint8_t> img(G::IMG, 0);
  // S_NB padded with a zero row and column, split into bf16 hi and lo (round to nearest even)
  auto bf16 = [](float v) -> uint16_t {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
  };
  auto unbf = [](uint16_t h) -> float {
    const uint32_t u = uint32_t(h) << 16;
    float v;
    std::memcpy(&v, &u, 4);
    return v;
  };
  const double sc = std::sqrt(2.0 / (n1 + 1)), pi = 3.14159265358979323846;
  std::vector<uint16_t> hi(NB * NB, 0), lo(NB * NB, 0);
  for (int p = 0; p < n1; ++p)
    for (int i = 0; i < n1; ++i) {
      const float v = float(sc * std::sin(pi * double(p + 1) * double(i + 1) / double(n1 + 1)));
      const uint16_t h = bf16(v);
      hi[p * NB + i] = h;
      lo[p * NB + i] = bf16(v - unbf(h));
    }
  auto put = [&](int base, int R, int r, int k, uint16_t v) { std::memcpy(&img[base + off_kmajor(R, r, k)], &v, 2); };
  // S_128: block-diagonal copies of S_NB
  for (int r = 0; r < 128; ++r)
    for (int k = 0; k < 128; ++k) {
      if (r / NB != k / NB) continue;
      put(G::oSAh, 128, r, k, hi[(r % NB) * NB + k % NB]);
      put(G::oSAl, 128, r, k, lo[(r % NB) * NB + k % NB]);
    }
  if (NB < 128)
    for (int r = 0; r < NB; ++r)
      for (int k = 0; k < NB; ++k) {
        put(G::oSBh, NB, r, k, hi[r * NB + k]);
        put(G::oSBl, NB, r, k, lo[r * NB + k]);
      }
  // t_i = 1 - cos th_i = 2 sin^2(th_i / 2); the padding mode takes 1 (cos = 0: a positive lambda)
  for (int i = 0; i < NB; ++i) {
    const double s = std::sin(pi * double(i + 1) / (2.0 * (n1 + 1)));
    const float t = i < n1 ? float(2.0 * s * s) : 1.0f;
    std::memcpy(&img[G::oT + 4 * i], &t, 4);
  }
  return img;
}

// eigenvalue coefficients in the cancellation-free form (t = 1 - cos th):
// lambda = (d + 4e + 4c) - (2e + 4c)(t_i + t_j) + 4c t_i t_j
static void lambda_coefs(double d, double e, double c, float* l0, float* l1, float* l2) {
  *l0 = float(d + 4.0 * e + 4.0 * c);
  *l1 = float(-(2.0 * e + 4.0 * c));
  *l2 = float(4.0 * c);
}

template <int NB, int PREC>
cudaError_t launch_nb(const float* b, float* x, int64_t B, const void* img, double d, double e, double c, float* acc,
                      int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st, VColumns cols, const SpecMulti& sm,
                      const SpecScale& sc) {
  using G = SpecGeo<NB>;
  auto k = spectral_mean_kernel<NB, PREC>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  if (err != cudaSuccess) return err;
  float l0, l1, l2;
  lambda_coefs(d, e, c, &l0, &l1, &l2);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned((B + G::CPT - 1) / G::CPT * sm.ng));
  cfg.blockDim = dim3(kSpecThreads);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_take_fence(st) ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, k, b, x, B, static_cast<const uint8_t*>(img), l0, l1, l2, acc, acc_ss, acc_L,
                            acc_col0, cols, sm, sc);
}

bool spectral_mean_supported(int n1) { return n1 == 63 || n1 == 127; }

size_t spectral_image_bytes(int n1) {
  if (n1 == 63) return size_t(SpecGeo<64>::IMG);
  if (n1 == 127) return size_t(SpecGeo<128>::IMG);
  return 0;
}

std::vector<uint8_t> spectral_image(int n1) {
  if (n1 == 63) return build_image<64>(n1);
  if (n1 == 127) return build_image<128>(n1);
  return {};
}

static cudaError_t launch_spectral_any(const float* b, float* x, int64_t B, int n1, const void* img, double d,
                                       double e, double c, float* acc, int64_t acc_ss, int acc_L, int acc_col0,
                                       cudaStream_t st, VColumns cols, int prec, const SpecMulti& sm,
                                       const SpecScale& sc = SpecScale());

cudaError_t launch_spectral_mean(const float* b, float* x, int64_t B, int n1, const void* img, double d, double e,
                                 double c, float* acc, int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st,
                                 VColumns cols, int prec) {
  static const SpecMulti solo{};
  return launch_spectral_any(b, x, B, n1, img, d, e, c, acc, acc_ss, acc_L, acc_col0, st, cols, prec, solo);
}

cudaError_t launch_spectral_mean_group(const float* const* b, float* const* x, float* const* acc,
                                       const double (*stencil)[3], int ng, int64_t B, int n1, const void* img,
                                       int64_t acc_ss, int acc_L, int acc_col0, cudaStream_t st, VColumns cols) {
  if (ng < 1 || ng > kMaxGroup) return cudaErrorInvalidValue;
  SpecMulti sm{};
  sm.ng = ng;
  for (int g = 0; g < ng; ++g) {
    if ((acc[g] != nullptr) != (acc[0] != nullptr)) return cudaErrorInvalidValue;
    sm.b[g] = b[g]; sm.x[g] = x[g]; sm.acc[g] = acc[g];
    lambda_coefs(stencil[g][0], stencil[g][1], stencil[g][2], &sm.l0[g], &sm.l1[g], &sm.l2[g]);
  }
  return launch_spectral_any(b[0], x[0], B, n1, img, stencil[0][0], stencil[0][1], stencil[0][2], acc[0], acc_ss,
                             acc_L, acc_col0, st, cols, 0, sm);
}

cudaError_t launch_spectral_mass(const float* B, float* X, int64_t ncols, int n1, const void* img, double h2_36,
                                 const SpecScale& sc, cudaStream_t st) {
  static const SpecMulti solo{};
  return launch_spectral_any(B, X, ncols, n1, img, 16.0 * h2_36, 4.0 * h2_36, h2_36, nullptr, 0, 1, 0, st,
                             VColumns(), 0, solo, sc);
}

static cudaError_t launch_spectral_any(const float* b, float* x, int64_t B, int n1, const void* img, double d,
                                       double e, double c, float* acc, int64_t acc_ss, int acc_L, int acc_col0,
                                       cudaStream_t st, VColumns cols, int prec, const SpecMulti& sm,
                                       const SpecScale& sc) {
  if (B == 0) return cudaSuccess;
  if (!spectral_mean_supported(n1) || img == nullptr || (reinterpret_cast<uintptr_t>(img) & 15) || prec < 0 ||
      prec > 2)
    return cudaErrorInvalidValue;
  const int NB = n1 + 1, CPT = 128 / NB;
  const double tiles = double((B + CPT - 1) / CPT) * sm.ng;
  // tensor work: per tile 3 - prec bf16 products for each of G1, G3 (128 x NB x NB) and G2, G4
  // (128 x 128 x NB)
  const double n0 = double(n1) * n1;
  ProfScope ps(KK_MEAN_EXACT, st, 4.0 * double(B) * sm.ng * n0 * (acc ? 3 : 2),
               tiles * double(3 - prec) * 2.0 * 2.0 * 128.0 * NB * (double(NB) + 128.0));
  cudaError_t err;
  if (prec != 0) return cudaErrorInvalidValue;     // only the exact form is built (see the kernel)
  err = n1 == 63 ? launch_nb<64, 0>(b, x, B, img, d, e, c, acc, acc_ss, acc_L, acc_col0, st, cols, sm, sc)
                 : launch_nb<128, 0>(b, x, B, img, d, e, c, acc, acc_ss, acc_L, acc_col0, st, cols, sm, sc);
  add_launches(1);
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t spectral_take_error(bool* failed, cudaStream_t st) {
  static int* host = nullptr;
  if (host == nullptr) {
    cudaError_t e = cudaMallocHost(&host, sizeof(int));
    if (e != cudaSuccess) return e;
  }
  static const int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(host, g_spec_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *failed = *host != 0;
  if (*failed) {
    e = cudaMemcpyToSymbolAsync(g_spec_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e;
}

}  // namespace sgoc
