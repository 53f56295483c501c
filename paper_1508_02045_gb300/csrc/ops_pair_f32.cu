// Launchers of the FP32 kernels specialised at compile time for two-stage plans (pair_fft.cuh),
// in a translation unit of their own so that they compile in parallel with the rest.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "ops.h"
#include "pair_fft.cuh"
#include "pcg_pot.cuh"

namespace hom {

bool pair_plan_f32(const AxisPlan& P) {
  if (P.nst != 2) return false;
#define HOM_PAIR_IS(R1_, R2_) \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) return true;
  HOM_PAIR_PLANS(HOM_PAIR_IS)
#undef HOM_PAIR_IS
  return false;
}

#define HOM_SET_SMEM(kern)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                          cap);                                               \
    if (e_ != cudaSuccess) return e_;                                                         \
  } while (0)

// ---------------------------------------------------------------------------------------
// TMA tensor maps and the device counter of TMA waits that ran out
// ---------------------------------------------------------------------------------------
constexpr int kTmaDevices = 64;
static __device__ unsigned g_tma_wait_errors;

static unsigned* tma_error_counter() {
  static unsigned* addr[kTmaDevices] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kTmaDevices) return nullptr;
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tma_wait_errors) == cudaSuccess) addr[dev] = (unsigned*)p;
  }
  return addr[dev];
}

unsigned tma_wait_errors(bool reset) {
  unsigned* p = tma_error_counter();
  if (p == nullptr) return 0;
  unsigned v = 0;
  if (cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  if (reset && v != 0) cudaMemset(p, 0, sizeof v);
  return v;
}

using TmaEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static TmaEncodeFn tma_encoder() {
  static const TmaEncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<TmaEncodeFn>(p);
  }();
  return fn;
}

bool tma_map_3d(CUtensorMap* map, const void* base, long long C, long long rows,
                long long batches, long long es, long long bs, int box_c, int box_rows) {
  constexpr long long el = 8;
  const TmaEncodeFn enc = tma_encoder();
  if (enc == nullptr) return false;
  if (((uintptr_t)base & 15) != 0 || (es * el) % 16 != 0 || (bs * el) % 16 != 0) return false;
  if ((box_c * el) % 16 != 0 || box_c > 256 || box_rows > 256 || box_c < 1 || box_rows < 1)
    return false;
  if (C < 1 || rows < 1 || batches < 1 || es < C || bs < es * rows) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)rows, (cuuint64_t)batches};
  const cuuint64_t strides[2] = {(cuuint64_t)(es * el), (cuuint64_t)(bs * el)};
  const cuuint32_t box[3] = {(cuuint32_t)box_c, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// bytes announced on top of each TMA tile copy (hom_debug_tma_stall)
static unsigned g_tma_extra_tx = 0;
void tma_debug_stall(bool on) { g_tma_extra_tx = on ? 16u : 0u; }

// the TMA-staged strided pass is used unless HOM_PAIR_TMA=0
static bool pair_tma_enabled() {
  static const bool on = [] {
    const char* e = getenv("HOM_PAIR_TMA");
    return e == nullptr || e[0] != '0';
  }();
  return on;
}

// persistent grid of a TMA-staged kernel: its resident CTAs on every SM
template <typename K>
static int persistent_ctas(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess)
    per = 0;
  return std::max(1, per) * std::max(1, sms);
}

// resident CTAs of the TMA-staged strided kernel of a plan on the current device (set by
// pair_prepare_f32, before any stream capture)
template <int R1, int R2, bool INV>
static int& strided_tma_ctas() {
  static int v[kTmaDevices] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  return v[(unsigned)dev % kTmaDevices];
}

cudaError_t pair_prepare_f32(int cap) {
  using T = float;
  // this unit's copies of the register-DFT constants
  const cudaError_t e = upload_reg_tables();
  if (e != cudaSuccess) return e;
#define HOM_PAIR_SMEM(R1_, R2_)                                 \
  HOM_SET_SMEM((k_pair_strided<T, R1_, R2_, false>));           \
  HOM_SET_SMEM((k_pair_strided<T, R1_, R2_, true>));            \
  HOM_SET_SMEM((k_pair_strided_tma<T, R1_, R2_, false>));       \
  HOM_SET_SMEM((k_pair_strided_tma<T, R1_, R2_, true>));        \
  HOM_SET_SMEM((k_pair_proj<T, 2, PROJ_GAMMA, R1_, R2_>));      \
  HOM_SET_SMEM((k_pair_proj<T, 2, PROJ_EM, R1_, R2_>));         \
  HOM_SET_SMEM((k_pair_proj<T, 3, PROJ_GAMMA, R1_, R2_>));      \
  HOM_SET_SMEM((k_pair_proj<T, 3, PROJ_EM, R1_, R2_>));         \
  HOM_SET_SMEM((k_pair_proj_scalar<T, R1_, R2_, false>));       \
  HOM_SET_SMEM((k_pair_proj_scalar<T, R1_, R2_, true>));        \
  HOM_SET_SMEM((k_pair_strided2<T, R1_, R2_, false>));          \
  HOM_SET_SMEM((k_pair_strided2<T, R1_, R2_, true>));           \
  HOM_SET_SMEM((k_pair_line_fwd<T, 3, PRE_CG, R1_, R2_>));      \
  HOM_SET_SMEM((k_pair_line_fwd<T, 3, PRE_CG_DOT, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_CG_FUSED, R1_, R2_>)); \
  HOM_SET_SMEM((k_pair_line_fwd<T, 3, PRE_LINEAR, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_CG, R1_, R2_>));     \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_CHEB, R1_, R2_>));   \
  HOM_SET_SMEM((k_pair_line_inv<T, 3, POST_STORE, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_fwd<T, 6, PRE_CG_DOT, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_fwd<T, 6, PRE_LINEAR, R1_, R2_>));  \
  HOM_SET_SMEM((k_pair_line_inv<T, 6, POST_CG_FUSED, R1_, R2_>)); \
  HOM_SET_SMEM((k_pair_line_inv<T, 6, POST_CHEB, R1_, R2_>));
  HOM_PAIR_PLANS(HOM_PAIR_SMEM)
#undef HOM_PAIR_SMEM
#define HOM_PAIR_TMA_CTAS(R1_, R2_)                                                            \
  strided_tma_ctas<R1_, R2_, false>() =                                                        \
      persistent_ctas(k_pair_strided_tma<T, R1_, R2_, false>, pair_tc_strided<R2_>() * R2_,    \
                      pair_strided_tma_smem<T, R1_, R2_>());                                   \
  strided_tma_ctas<R1_, R2_, true>() =                                                         \
      persistent_ctas(k_pair_strided_tma<T, R1_, R2_, true>, pair_tc_strided<R2_>() * R2_,     \
                      pair_strided_tma_smem<T, R1_, R2_>());
  HOM_PAIR_PLANS(HOM_PAIR_TMA_CTAS)
#undef HOM_PAIR_TMA_CTAS
  tma_error_counter();
  tma_encoder();
#define HOM_POT_SMEM(R1_, R2_)                                  \
  HOM_SET_SMEM((k_pot_inv<T, R1_, R2_, POT_STEP>));             \
  HOM_SET_SMEM((k_pot_inv<T, R1_, R2_, POT_FIELD>));            \
  HOM_SET_SMEM((k_pot_fwd<T, R1_, R2_, POT_UPDATE>));           \
  HOM_SET_SMEM((k_pot_fwd<T, R1_, R2_, POT_INIT>));             \
  HOM_SET_SMEM((k_pot_line<T, 3, R1_, R2_>));
  HOM_PAIR_PLANS(HOM_POT_SMEM)
#undef HOM_POT_SMEM
  return cudaSuccess;
}

// ---- conjugate gradients in potential coordinates (pcg_pot.cuh) ----
void pot_inv_f32(int mode, const AxisPlan& P, cpx<float>* S, const cpx<float>* tw,
                 const ProjGeom& pg, const PotVecs<float>& V, const Scalars* sc, cudaStream_t st,
                 const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const bool prof = profiling();
#define HOM_POT_INV(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pot_tc_inv<R2_>();                                             \
    const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                     \
    const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + 2 * (TC + 1)));             \
    if (prof) prof_mark(KIND_POT_INV, st, true);                                               \
    if (mode == POT_FIELD)                                                                     \
      launch_pass(k_pot_inv<T, R1_, R2_, POT_FIELD>, grid, 2 * TC * R2_, sm, st, S, tw, pg, V, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pot_inv<T, R1_, R2_, POT_STEP>, grid, 2 * TC * R2_, sm, st, S, tw, pg, V, sc, reqs); \
    if (prof) prof_mark(KIND_POT_INV, st, false);                                              \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_POT_INV)
#undef HOM_POT_INV
}

void pot_fwd_f32(int mode, const AxisPlan& P, const cpx<float>* S, const cpx<float>* tw,
                 const ProjGeom& pg, const PotVecs<float>& V, Scalars* sc, double* partials,
                 unsigned* counter, cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const bool prof = profiling();
#define HOM_POT_FWD(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pot_tc_fwd<R2_>();                                             \
    const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                     \
    const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + 2 * (TC + 1)));             \
    if (prof) prof_mark(KIND_POT_FWD, st, true);                                               \
    if (mode == POT_INIT)                                                                      \
      launch_pass(k_pot_fwd<T, R1_, R2_, POT_INIT>, grid, pot_fwd_threads<R2_>(), sm, st, S, tw, pg, V, sc, partials, counter, reqs); \
    else                                                                                       \
      launch_pass(k_pot_fwd<T, R1_, R2_, POT_UPDATE>, grid, pot_fwd_threads<R2_>(), sm, st, S, tw, pg, V, sc, partials, counter, reqs); \
    if (prof) prof_mark(KIND_POT_FWD, st, false);                                              \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_POT_FWD)
#undef HOM_POT_FWD
}

int pot_line_f32(const AxisPlan& P, cpx<float>* S, const cpx<float>* tw, long long nlines,
                 long long scs, const MatView<float>& mat, Scalars* sc, double* partials,
                 cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const bool prof = profiling();
#define HOM_POT_LINE(R1_, R2_)                                                                 \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int LB = 2 * pair_lbp<3, R2_>();                                                 \
    const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                   \
    const size_t sm = PairFwdSmem<3, R1_, R2_>::bytes;                                         \
    constexpr int NT = pair_line_threads<3, R2_>();                                            \
    if (prof) prof_mark(KIND_POT_LINE, st, true);                                              \
    launch_pass(k_pot_line<T, 3, R1_, R2_>, grid, NT, sm, st, S, tw, nlines, scs, mat, sc,       \
                partials, reqs);                                                               \
    if (prof) prof_mark(KIND_POT_LINE, st, false);                                             \
    return (int)grid.x;                                                                        \
  }
  HOM_PAIR_PLANS(HOM_POT_LINE)
#undef HOM_POT_LINE
  return 0;
}

// Shared memory requested by a strided CTA of 128 threads or more: 39424 bytes a CTA with the
// driver's reserve, so that six no longer fit the SM (228 KiB) and five keep its 196 KiB
// configuration. The 243-point forward pass, whose registers allow six CTAs, ran 0.075 instead
// of 0.078 ms (averaged with the inverse pass) at five: six CTAs queue up on shared memory.
constexpr size_t kPairStridedMinSmem = 38400;

void pair_strided_f32(const AxisPlan& P, int inv, cpx<float>* S, const cpx<float>* tw,
                      long long C, long long es, long long bs, int batches, const Scalars* sc,
                      cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
#define HOM_PAIR_ST(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pair_tc_strided<R2_>();                                                 \
    CUtensorMap map;                                                                           \
    const long long ntc = (C + TC - 1) / TC, ntiles = ntc * batches;                          \
    if (reqs == nullptr && nreq == 1 && pair_tma_enabled() && ntiles < (1LL << 30) &&         \
        tma_map_3d(&map, S, C, R1_ * R2_, batches, es, bs, TC, R1_ * R2_)) {                  \
      constexpr size_t sm = pair_strided_tma_smem<T, R1_, R2_>();                              \
      auto kern = inv ? k_pair_strided_tma<T, R1_, R2_, true>                                  \
                      : k_pair_strided_tma<T, R1_, R2_, false>;                                \
      int& nc = inv ? strided_tma_ctas<R1_, R2_, true>() : strided_tma_ctas<R1_, R2_, false>(); \
      if (nc == 0) nc = persistent_ctas(kern, TC * R2_, sm);                                   \
      const int grid = (int)std::min<long long>(nc, ntiles);                                   \
      launch_pass(kern, dim3((unsigned)grid), TC * R2_, sm, st, map, S, tw, C, es, bs,         \
                  (int)ntc, (int)ntiles, sc, tma_error_counter(), g_tma_extra_tx);             \
      return;                                                                                  \
    }                                                                                          \
    const dim3 grid((unsigned)((C + TC - 1) / TC), (unsigned)batches, (unsigned)nreq);        \
    size_t sm = sizeof(cpx<T>) * (size_t)(R1_ * R2_) * (TC + 2);                                \
    if (TC * R2_ >= 128 && sm < kPairStridedMinSmem) sm = kPairStridedMinSmem;                 \
    if (inv)                                                                                   \
      launch_pass(k_pair_strided<T, R1_, R2_, true>, grid, TC * R2_, sm, st, S, tw, C, es, bs, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pair_strided<T, R1_, R2_, false>, grid, TC * R2_, sm, st, S, tw, C, es, bs, sc, reqs); \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_ST)
#undef HOM_PAIR_ST
}

void pair_strided2_f32(const AxisPlan& P, int inv, cpx<float>* S, const cpx<float>* tw,
                       long long C, long long es, long long bs, long long cs, int planes,
                       const Scalars* sc, cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
#define HOM_PAIR_ST2(R1_, R2_)                                                                 \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    constexpr int TC = pair_tc_strided<R2_>();                                                 \
    const dim3 grid((unsigned)((C + TC - 1) / TC), (unsigned)planes, (unsigned)nreq);         \
    const size_t sm = sizeof(cpx<T>) * (size_t)(R1_ * R2_) * (1 + 2 * (TC + 1));               \
    if (inv)                                                                                   \
      launch_pass(k_pair_strided2<T, R1_, R2_, true>, grid, 2 * TC * R2_, sm, st, S, tw, C, es, bs, cs, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pair_strided2<T, R1_, R2_, false>, grid, 2 * TC * R2_, sm, st, S, tw, C, es, bs, cs, sc, reqs); \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_ST2)
#undef HOM_PAIR_ST2
}

void pair_proj_f32(int D, int mode, bool two, const AxisPlan& P, cpx<float>* S,
                   const cpx<float>* tw, const ProjGeom& pg, const Scalars* sc, cudaStream_t st,
                   const ReqDesc<float>* reqs, int nreq) {
  using T = float;
#define HOM_PAIR_PJ_D(D_, R1_, R2_)                                                            \
  {                                                                                            \
    constexpr int TC = pair_tc_proj<D_, R2_>();                                                \
    const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                     \
    const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + D_ * (TC + 1)));        \
    if (mode == PROJ_EM)                                                                       \
      launch_pass(k_pair_proj<T, D_, PROJ_EM, R1_, R2_>, grid, D_ * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
    else                                                                                       \
      launch_pass(k_pair_proj<T, D_, PROJ_GAMMA, R1_, R2_>, grid, D_ * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
  }
#define HOM_PAIR_PJ(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    if (D == 2) {                                                                              \
      HOM_PAIR_PJ_D(2, R1_, R2_)                                                               \
    } else if (mode == PROJ_GAMMA) {                                                           \
      constexpr int TC = pair_tc_proj_scalar<R2_>();                                           \
      const dim3 grid((unsigned)((pg.C + TC - 1) / TC), 1, (unsigned)nreq);                   \
      const size_t sm = sizeof(cpx<T>) * ((size_t)(R1_ * R2_) * (1 + 2 * (TC + 1)));           \
      if (two)                                                                                 \
        launch_pass(k_pair_proj_scalar<T, R1_, R2_, true>, grid, 2 * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
      else                                                                                     \
        launch_pass(k_pair_proj_scalar<T, R1_, R2_, false>, grid, 2 * TC * R2_, sm, st, S, tw, pg, sc, reqs); \
    } else {                                                                                   \
      HOM_PAIR_PJ_D(3, R1_, R2_)                                                               \
    }                                                                                          \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_PJ)
#undef HOM_PAIR_PJ
#undef HOM_PAIR_PJ_D
}

int pair_line_fwd_f32(int D, int pre, const AxisPlan& P, const Fields<float>& f, cpx<float>* S,
                      const cpx<float>* tw, long long nlines, long long scs,
                      const MatView<float>& mat, Scalars* sc, const OpArgs& args,
                      double* partials, cudaStream_t st, const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const FastDiv fdn = make_fastdiv(P.n);
#define HOM_PAIR_LF_P(D_, PRE_, R1_, R2_)                                                      \
  launch_pass(k_pair_line_fwd<T, D_, PRE_, R1_, R2_>, grid, NT, sm, st, f, S, tw, nlines, scs, mat, sc, \
              args, fdn, partials, reqs)
#define HOM_PAIR_LF(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    if (D == 6) {                                                                              \
      constexpr int LB = 2 * pair_lbp<6, R2_>();                                               \
      const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                 \
      const size_t sm = PairFwdSmem<6, R1_, R2_>::bytes;                                       \
      constexpr int NT = pair_line_threads<6, R2_>();                                          \
      if (pre == PRE_CG_DOT) HOM_PAIR_LF_P(6, PRE_CG_DOT, R1_, R2_);                           \
      else HOM_PAIR_LF_P(6, PRE_LINEAR, R1_, R2_);                                             \
      return (int)grid.x;                                                                      \
    }                                                                                          \
    constexpr int LB = 2 * pair_lbp<3, R2_>();                                                 \
    const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                   \
    const size_t sm = PairFwdSmem<3, R1_, R2_>::bytes;                                         \
    constexpr int NT = pair_line_threads<3, R2_>();                                            \
    if (pre == PRE_CG) HOM_PAIR_LF_P(3, PRE_CG, R1_, R2_);                                     \
    else if (pre == PRE_CG_DOT) HOM_PAIR_LF_P(3, PRE_CG_DOT, R1_, R2_);                        \
    else HOM_PAIR_LF_P(3, PRE_LINEAR, R1_, R2_);                                               \
    return (int)grid.x;                                                                        \
  }
  HOM_PAIR_PLANS(HOM_PAIR_LF)
  return 0;
#undef HOM_PAIR_LF
#undef HOM_PAIR_LF_P
}

void pair_line_inv_f32(int D, int post, const AxisPlan& P, const cpx<float>* S,
                       const Fields<float>& f, const cpx<float>* tw, long long nlines,
                       long long scs, const MatView<float>& mat, Scalars* sc, const OpArgs& args,
                       double* partials, unsigned* counter, int negate, cudaStream_t st,
                       const ReqDesc<float>* reqs, int nreq) {
  using T = float;
  const FastDiv fdn = make_fastdiv(P.n);
#define HOM_PAIR_LI_P(D_, POST_, R1_, R2_)                                                     \
  launch_pass(k_pair_line_inv<T, D_, POST_, R1_, R2_>, grid, NT, sm, st, S, f, tw, nlines, scs, mat, \
              sc, args, partials, counter, negate, fdn, reqs)
#define HOM_PAIR_LI(R1_, R2_)                                                                  \
  if (P.radix[0] == R1_ && P.radix[1] == R2_) {                                                \
    if (D == 6) {                                                                              \
      constexpr int LB = 2 * pair_lbp<6, R2_>();                                               \
      const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                 \
      const size_t sm = PairFwdSmem<6, R1_, R2_>::bytes;                                       \
      constexpr int NT = pair_line_threads<6, R2_>();                                          \
      if (post == POST_CG_FUSED) HOM_PAIR_LI_P(6, POST_CG_FUSED, R1_, R2_);                    \
      else HOM_PAIR_LI_P(6, POST_CHEB, R1_, R2_);                                              \
      return;                                                                                  \
    }                                                                                          \
    constexpr int LB = 2 * pair_lbp<3, R2_>();                                                 \
    const dim3 grid((unsigned)((nlines + LB - 1) / LB), 1, (unsigned)nreq);                   \
    const size_t sm = PairFwdSmem<3, R1_, R2_>::bytes;                                         \
    constexpr int NT = pair_line_threads<3, R2_>();                                            \
    if (post == POST_CG) HOM_PAIR_LI_P(3, POST_CG, R1_, R2_);                                  \
    else if (post == POST_CG_FUSED) HOM_PAIR_LI_P(3, POST_CG_FUSED, R1_, R2_);                 \
    else if (post == POST_CHEB) HOM_PAIR_LI_P(3, POST_CHEB, R1_, R2_);                         \
    else HOM_PAIR_LI_P(3, POST_STORE, R1_, R2_);                                               \
    return;                                                                                    \
  }
  HOM_PAIR_PLANS(HOM_PAIR_LI)
#undef HOM_PAIR_LI
#undef HOM_PAIR_LI_P
}

}  // namespace hom
