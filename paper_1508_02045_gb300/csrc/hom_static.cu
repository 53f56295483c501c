// hom_apply_static: one operator application that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns every byte of device
// memory through its own allocator or a fixed budget, a plugin loaded into such an
// application, or a latency-critical loop that must not pay for cudaMalloc/cudaFree (both can
// synchronise the whole device and stall unrelated streams). For them this file keeps the
// work memory of the operator (half spectrum, twiddle tables, coefficient table) in one
// file-scope __device__ array of HOM_STATIC_SCRATCH_BYTES, which every GPU that loads the
// library holds until the process exits. The caller passes inputs and outputs only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hom.h"
#include "ops.h"
#include "passes.cuh"
#include "problem.h"

using namespace hom;

namespace {

constexpr size_t kTwBytes = 64 * 1024;                 // three twiddle tables (<= 1023 each)
constexpr size_t kTabBytes = 512 * 1024;               // coefficient table (<= 65536 doubles)
constexpr size_t kSpecOff = kTwBytes + kTabBytes;      // half spectrum after both
static_assert(3 * kMaxAxis * sizeof(cpx<double>) <= kTwBytes, "twiddle region too small");

}  // namespace

// The scratch itself. Host code must not use this name as an address: it is a host-side
// stand-in for the device symbol. The device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_hom_scratch[HOM_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_base[kMaxDevices] = {};

// Per-device set-up, once, with that device current: resolve the scratch address, upload the
// DFT constants and raise the kernels' shared-memory limits. No allocation.
int static_setup(int dev, unsigned char** base) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (g_static_base[dev] != nullptr) {
    *base = g_static_base[dev];
    return HOM_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_hom_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return HOM_ERR_CUDA;
  }
  if (Ops<double>::upload_constants() != cudaSuccess || Ops<double>::prepare(3) != cudaSuccess) {
    cudaGetLastError();
    return HOM_ERR_CUDA;
  }
  g_static_base[dev] = static_cast<unsigned char*>(p);
  *base = g_static_base[dev];
  return HOM_OK;
}

// Values written into the scratch by a kernel whose parameters carry them: a launch copies
// its parameters when it is enqueued, so the call needs no host staging buffer that must
// outlive it and no pageable host-to-device copy (which would wait for the stream's earlier
// work before returning).
constexpr int kFillChunk = 496;  // doubles per launch (kernel parameters stay under 4 KiB)
struct FillChunk {
  int count;
  double v[kFillChunk];
};

__global__ void k_static_fill(double* __restrict__ dst, FillChunk c) {
  for (int i = threadIdx.x; i < c.count; i += blockDim.x) dst[i] = c.v[i];
}

bool fill_device(double* dst, const double* src, size_t n, cudaStream_t st) {
  for (size_t o = 0; o < n; o += kFillChunk) {
    FillChunk c;
    c.count = (int)std::min<size_t>(kFillChunk, n - o);
    std::memcpy(c.v, src + o, sizeof(double) * (size_t)c.count);
    k_static_fill<<<1, 128, 0, st>>>(dst + o, c);
    ++launch_counter();
  }
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace

extern "C" int hom_apply_static(int d, const int* N, const void* phase_dev, int index_bytes,
                                const double* table, int nphase, int op, const double* E,
                                const double* x_dev, double* y_dev, void* stream) {
  if ((d != 2 && d != 3) || !N || !phase_dev || !table || !x_dev || !y_dev) return HOM_ERR_INVALID;
  if (index_bytes != 1 && index_bytes != 2) return HOM_ERR_INVALID;
  if (nphase < 1 || (index_bytes == 1 && nphase > 256)) return HOM_ERR_INVALID;
  if (op < HOM_OP_AFFINE || op > HOM_OP_EM || (op == HOM_OP_AFFINE && !E)) return HOM_ERR_INVALID;
  PassGeom g{};
  AxisPlan plan[3]{};
  g.D = d;
  g.nodes = 1;
  for (int a = 0; a < d; ++a) {
    if (!hom::detail::plan_axis(N[a], hom::detail::reg_rmax<double>(), &plan[a]))
      return HOM_ERR_INVALID;
    g.n[a] = N[a];
    g.nodes *= N[a];
  }
  for (int a = d; a < 3; ++a) g.n[a] = 1;
  const int nl = N[d - 1];
  g.nh = (nl + 1) / 2;
  g.nlines = g.nodes / nl;
  g.scs = g.nlines * g.nh;

  // ---- size limits of the static scratch ----
  const size_t spec_bytes = sizeof(cpx<double>) * (size_t)d * (size_t)g.scs;
  const bool iso_table = [&] {
    for (int p = 0; p < nphase; ++p)
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          const double v = table[(size_t)p * d * d + i * d + j];
          if ((i != j && v != 0.0) || (i == j && v != table[(size_t)p * d * d])) return false;
        }
    return true;
  }();
  const size_t tab_bytes = sizeof(double) * (size_t)nphase * (iso_table ? 1 : d * d);
  if (kSpecOff + spec_bytes > (size_t)HOM_STATIC_SCRATCH_BYTES || tab_bytes > kTabBytes)
    return HOM_ERR_SCRATCH;

  // ---- coefficients: SPD phases and the bounds c_A, C_A (eq. (A)) ----
  double cA = 1e300, CA = -1e300;
  std::vector<double> tab;
  for (int p = 0; p < nphase; ++p) {
    double lo, hi;
    if (!hom::detail::spd_eigs(table + (size_t)p * d * d, d, &lo, &hi)) return HOM_ERR_INVALID;
    cA = std::min(cA, lo);
    CA = std::max(CA, hi);
    if (iso_table) tab.push_back(table[(size_t)p * d * d]);
  }
  if (!iso_table) tab.assign(table, table + (size_t)nphase * d * d);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HOM_ERR_CUDA;
  unsigned char* base = nullptr;
  int rc = static_setup(dev, &base);
  if (rc != HOM_OK) return rc;

  // ---- launch geometry (the default budget of hom_create) ----
  if (!Ops<double>::plan_geometry(d, N, plan, 110 * 1024, kThreads, &g))
    return HOM_ERR_UNSUPPORTED;

  // ---- twiddles (the long-double tables of hom_create) and table into the scratch, by
  // kernels on the caller's stream ----
  cudaStream_t st = (cudaStream_t)stream;
  cpx<double>* tw[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < d; ++a) {
    tw[a] = reinterpret_cast<cpx<double>*>(base) + (size_t)a * kMaxAxis;
    const std::vector<cpx<double>> tw_h = hom::detail::twiddles<double>(N[a]);
    if (!fill_device(reinterpret_cast<double*>(tw[a]), &tw_h[0].x, 2 * tw_h.size(), st))
      return HOM_ERR_CUDA;
  }
  double* tab_dev = reinterpret_cast<double*>(base + kTwBytes);
  cpx<double>* S = reinterpret_cast<cpx<double>*>(base + kSpecOff);
  if (!fill_device(tab_dev, tab.data(), tab.size(), st)) return HOM_ERR_CUDA;

  // ---- one application: the same passes as hom_apply ----
  MatView<double> mat{};
  mat.kind = iso_table ? MAT_PHASE_ISO : MAT_PHASE_TENSOR;
  mat.ph8 = index_bytes == 1 ? static_cast<const uint8_t*>(phase_dev) : nullptr;
  mat.ph16 = index_bytes == 2 ? static_cast<const uint16_t*>(phase_dev) : nullptr;
  mat.table = tab_dev;
  ProjGeom pg{};
  pg.C = g.scs / N[0];
  pg.cs = g.scs;
  pg.n1 = d == 3 ? N[1] : 1;
  pg.nh = g.nh;
  pg.fdnh = make_fastdiv(g.nh);
  for (int a = 0; a < 3; ++a) pg.hw[a] = a < d ? (N[a] - 1) / 2 : 0;
  pg.scale = 1.0 / (double)g.nodes;
  OpArgs args{};
  for (int a = 0; a < d; ++a) args.E[a] = E ? E[a] : 0.0;
  args.omega = std::sqrt(cA * CA);
  Fields<double> f{};
  f.xin = x_dev;
  f.out = y_dev;
  f.cs = g.nodes;
  const int pre = op == HOM_OP_AFFINE ? PRE_AFFINE : op == HOM_OP_LINEAR ? PRE_LINEAR
                : op == HOM_OP_PROJECT ? PRE_IDENT : PRE_EM;
  const int mode = op == HOM_OP_EM ? PROJ_EM : PROJ_GAMMA;
  Ops<double>::line_fwd(g, pre, f, S, plan[d - 1], tw[d - 1], d, mat, nullptr, args, st);
  if (d == 3) Ops<double>::strided(g, 1, 0, S, plan[1], tw[1], d, nullptr, st);
  Ops<double>::proj(g, mode, S, plan[0], tw[0], pg, nullptr, st);
  if (d == 3) Ops<double>::strided(g, 1, 1, S, plan[1], tw[1], d, nullptr, st);
  Ops<double>::line_inv(g, POST_STORE, S, f, plan[d - 1], tw[d - 1], d, mat, nullptr, args,
                        nullptr, nullptr, 0, st);
  if (cudaGetLastError() != cudaSuccess) return HOM_ERR_CUDA;
  return HOM_OK;
}
