// Batched iterations of same-shape solves (hom_batch) and the continuous-batching request
// server built on them (hom_server). Both are build extensions around Algorithms 1-4: every
// request runs exactly the solver steps of a solo hom_solve, with its own buffers, device
// scalars and reduction partials, so its result does not depend on what it is batched with.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <tuple>
#include <type_traits>
#include <vector>

#include "problem.h"

using namespace hom;
using namespace hom::detail;

namespace {

// ---------------------------------------------------------------------------------------
// per-request descriptors of the batched launches
// ---------------------------------------------------------------------------------------
ReqDesc<double> desc64(hom_problem* P) {
  ReqDesc<double> r{};
  r.S = (cpx<double>*)P->S;
  r.mat = P->e64.mat;
  r.sc = P->d_sc;
  r.partials = P->partials;
  r.counter = P->counter;
  r.ff.cs = r.fi.cs = P->nodes;
  double* x = P->vec[0];
  double* rr = P->vec[2];
  double* p = P->vec[3];
  double* q = P->vec[4];
  switch (P->sv.solver) {
    case HOM_RICHARDSON:  // x_m / x_{m-1} alternate between vec[0] and vec[1]
      r.ff.x = x;
      r.fi.x = x;
      break;
    case HOM_CG:
      r.ff.xin = rr;
      r.ff.p = p;
      r.fi.out = q;
      r.fi.p = p;
      r.fi.x = x;
      r.fi.r = rr;
      break;
    case HOM_CHEBYSHEV:
      r.ff.xin = p;
      r.fi.p = p;
      r.fi.r = rr;
      r.fi.x = x;
      break;
    default:  // Eyre-Milton
      r.ff.xin = x;
      r.fi.x = x;
      break;
  }
  return r;
}

// inner FP32 solve of the iterative refinement (CG or Chebyshev on the FP32 operator)
ReqDesc<float> desc32(hom_problem* P) {
  ReqDesc<float> r{};
  r.S = (cpx<float>*)P->S;
  r.mat = P->e32.mat;
  r.sc = P->d_sc2;
  r.partials = P->partials;
  r.counter = P->counter;
  r.ff.cs = r.fi.cs = P->nodes;
  float* x = P->fvec[0];
  float* rr = P->fvec[1];
  float* p = P->fvec[2];
  float* q = P->fvec[3];
  if (P->sv.pot) {  // CG in potential coordinates: u, r, p as one-component half spectra
    r.fi.x = x;
    r.fi.r = rr;
    r.fi.p = p;
    return r;
  }
  if (P->sv.solver == HOM_CG) {
    r.ff.xin = rr;
    r.ff.p = p;
    r.fi.out = q;
    r.fi.p = p;
    r.fi.x = x;
    r.fi.r = rr;
  } else {
    r.ff.xin = p;
    r.fi.p = p;
    r.fi.r = rr;
    r.fi.x = x;
  }
  return r;
}

// placeholder descriptor of an empty slot: its scalars say "stopped", so every CTA of that
// slot returns at entry and never dereferences the other (null) pointers
template <typename T>
ReqDesc<T> idle_desc(Scalars* idle) {
  ReqDesc<T> r{};
  r.sc = idle;
  return r;
}

// One batched step of the solver `solver` over n descriptors (Algorithms 1-4; for refinement
// the FP32 inner step). Geometry from the engine of a representative problem.
template <typename T>
void batch_step(const Engine<T>& E, int solver, const ReqDesc<T>* reqs, int n, int red_grid,
                long long nodes, int d, cudaStream_t st, bool pot = false) {
  if (pot) {  // the FP32 inner CG or Chebyshev in potential coordinates (buffers from the
              // descriptors)
    E.pot_step(PotVecs<T>{}, nullptr, nullptr, nullptr, nullptr, st, reqs, n,
               solver == HOM_CHEBYSHEV);
    return;
  }
  switch (solver) {
    case HOM_RICHARDSON:
      E.apply_batch(PRE_AFFINE, PROJ_GAMMA, POST_RICH, reqs, n, st);
      break;
    case HOM_CG:  // the fused step of hom_solve (vector update inside the operator passes)
      E.apply_batch(PRE_CG_DOT, PROJ_GAMMA, POST_CG_FUSED, reqs, n, st);
      break;
    case HOM_CHEBYSHEV:
      E.apply_batch(PRE_LINEAR, PROJ_GAMMA, POST_CHEB, reqs, n, st);
      break;
    default:
      E.apply_batch(PRE_EM, PROJ_EM, POST_EM, reqs, n, st);
      break;
  }
}

__global__ void k_gather_done(const Scalars* const* sc, int n, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sc[i] != nullptr ? sc[i]->done : 1;
}

}  // namespace

// ===========================================================================================
// hom_batch
// ===========================================================================================
struct hom_batch {
  std::vector<hom_problem*> m;
  int solver = 0;
  bool refined = false;
  cudaStream_t stream = nullptr;
  ReqDesc<double>* d64 = nullptr;
  ReqDesc<float>* d32 = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  long long graph_launches = 0;  // kernels in one replay of the graph
  bool pot = false;  // refined CG members run their inner solves in potential coordinates
};

namespace {

int batch_capture(hom_batch* B, int steps) {
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  hom_problem* P0 = B->m[0];
  const int n = (int)B->m.size();
  cudaGraph_t g = nullptr;
  const bool prof = profiling();
  if (prof) hom_profile_enable(0);
  if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    if (prof) hom_profile_enable(1);
    return HOM_ERR_CUDA;
  }
  const long long c0 = launch_counter();
  for (int k = 0; k < steps; ++k) {
    if (B->refined)
      batch_step<float>(P0->e32, B->solver, B->d32, n, P0->red_grid, P0->nodes, P0->d, B->stream,
                        B->pot);
    else
      batch_step<double>(P0->e64, B->solver, B->d64, n, P0->red_grid, P0->nodes, P0->d, B->stream);
  }
  // the kernels recorded into the graph run once per replay: count them there
  B->graph_launches = launch_counter() - c0;
  launch_counter() = c0;
  const cudaError_t e = cudaStreamEndCapture(B->stream, &g);
  if (prof) hom_profile_enable(1);
  if (e != cudaSuccess) return HOM_ERR_CUDA;
  const cudaError_t e2 = cudaGraphInstantiate(&B->graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    B->graph = nullptr;
    return HOM_ERR_CUDA;
  }
  B->graph_steps = steps;
  return HOM_OK;
}

}  // namespace

extern "C" int hom_batch_create(hom_problem* const* problems, int count, hom_batch** out) {
  if (!problems || count < 1 || !out) return HOM_ERR_INVALID;
  *out = nullptr;
  hom_problem* P0 = problems[0];
  if (!P0 || !P0->sv.active) return HOM_ERR_INVALID;
  for (int i = 0; i < count; ++i) {
    hom_problem* P = problems[i];
    if (!P || !P->sv.active || P->sv.solver != P0->sv.solver || P->d != P0->d ||
        P->precision != P0->precision || P->integration != P0->integration ||
        P->stream != P0->stream || P->device != P0->device || P->sv.pot != P0->sv.pot)
      return HOM_ERR_INVALID;
    for (int a = 0; a < P->d; ++a)
      if (P->M[a] != P0->M[a] || P->N[a] != P0->N[a]) return HOM_ERR_INVALID;
  }
  auto* B = new hom_batch();
  B->m.assign(problems, problems + count);
  B->solver = P0->sv.solver;
  B->refined = P0->sv.refined;
  B->pot = P0->sv.pot;
  B->stream = P0->stream;
  if (B->refined) {
    std::vector<ReqDesc<float>> h;
    for (auto* P : B->m) h.push_back(desc32(P));
    if (alloc((void**)&B->d32, sizeof(ReqDesc<float>) * h.size())) { delete B; return HOM_ERR_OOM; }
    cudaMemcpy(B->d32, h.data(), sizeof(ReqDesc<float>) * h.size(), cudaMemcpyHostToDevice);
  } else {
    std::vector<ReqDesc<double>> h;
    for (auto* P : B->m) h.push_back(desc64(P));
    if (alloc((void**)&B->d64, sizeof(ReqDesc<double>) * h.size())) { delete B; return HOM_ERR_OOM; }
    cudaMemcpy(B->d64, h.data(), sizeof(ReqDesc<double>) * h.size(), cudaMemcpyHostToDevice);
  }
  if (check_last()) {
    hom_batch_destroy(B);
    return HOM_ERR_CUDA;
  }
  *out = B;
  return HOM_OK;
}

extern "C" int hom_batch_iterate(hom_batch* B, int iterations, int use_graph, int* all_done) {
  if (!B || iterations < 0) return HOM_ERR_INVALID;
  hom_problem* P0 = B->m[0];
  const int n = (int)B->m.size();
  // graphs need a capturable (non-default) stream; on the default stream launch directly
  if (use_graph && iterations > 0 && B->stream != nullptr) {
    const int steps = std::min(iterations, 8);
    if (!B->graph || B->graph_steps != steps) {
      int rc = batch_capture(B, steps);
      if (rc) return rc;
    }
    int done_steps = 0;
    while (done_steps + B->graph_steps <= iterations) {
      HOM_CUDA(cudaGraphLaunch(B->graph, B->stream));
      launch_counter() += B->graph_launches;
      done_steps += B->graph_steps;
    }
    for (; done_steps < iterations; ++done_steps) {
      if (B->refined)
        batch_step<float>(P0->e32, B->solver, B->d32, n, P0->red_grid, P0->nodes, P0->d, B->stream,
                        B->pot);
      else
        batch_step<double>(P0->e64, B->solver, B->d64, n, P0->red_grid, P0->nodes, P0->d, B->stream);
    }
  } else {
    for (int k = 0; k < iterations; ++k) {
      if (B->refined)
        batch_step<float>(P0->e32, B->solver, B->d32, n, P0->red_grid, P0->nodes, P0->d, B->stream,
                        B->pot);
      else
        batch_step<double>(P0->e64, B->solver, B->d64, n, P0->red_grid, P0->nodes, P0->d, B->stream);
    }
  }
  for (auto* P : B->m) P->sv.issued += iterations;
  int rc = check_last();
  if (rc) return rc;
  if (all_done) {
    int all = 1;
    for (auto* P : B->m) {
      if (B->refined) {
        if (P->sv.finished) continue;
        if ((rc = poll(P, P->d_sc2))) return rc;
        if (P->h_sc->done && (rc = refine_outer_update(P))) return rc;
        if (!P->sv.finished) all = 0;
      } else {
        if ((rc = poll(P, P->d_sc))) return rc;
        const int cap = P->sv.maxit + (P->sv.solver == HOM_RICHARDSON ? 1 : 0);
        if (!P->h_sc->done && P->sv.issued < cap) all = 0;
      }
    }
    *all_done = all;
  }
  return HOM_OK;
}

extern "C" void hom_batch_destroy(hom_batch* B) {
  if (!B) return;
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->d64) cudaFree(B->d64);
  if (B->d32) cudaFree(B->d32);
  delete B;
}

// ===========================================================================================
// hom_server: continuous batching of heterogeneous requests
// ===========================================================================================
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct ServerReq {
  long long id = 0;
  hom_request req{};
  std::vector<unsigned char> data;   // owned copy of the coefficient data (host)
  std::vector<double> table;
  size_t bytes = 0;                  // device bytes charged against the budget
  hom_problem* P = nullptr;
  int bucket = -1, slot = -1;
  Clock::time_point t_submit, t_admit;
};

// components of a request's fields: d, or d (d + 1) / 2 for a stiffness material
int req_nc(const hom_request& r) {
  return r.material.kind == HOM_A_STIFFNESS ? r.d * (r.d + 1) / 2 : r.d;
}

// a bucket: same grid, component count, integration, precision and solver; fixed-capacity
// slots
struct Bucket {
  int d = 0, nc = 0, M[3] = {1, 1, 1}, N[3] = {1, 1, 1};
  int integration = 0, precision = 0, solver = 0;
  int cap = 0;
  std::vector<ServerReq*> slots;
  Engine<double>* e64 = nullptr;  // plans and launch geometry of the bucket's shape
  Engine<float>* e32 = nullptr;
  long long nodes = 0;
  int red_grid = 0;
  ReqDesc<double>* d64 = nullptr;
  ReqDesc<float>* d32 = nullptr;
  const Scalars** d_sc = nullptr;  // per-slot scalars for the done-flag gather
  int* d_done = nullptr;
  int* h_done = nullptr;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  long long graph_launches = 0;  // kernels in one replay of the graph
  cudaStream_t stream = nullptr;  // the bucket's own stream: buckets overlap on the device
  int inner_form = 0;             // hom_opts.inner_form of its requests
  bool pot = false;               // their FP32 inner CG runs in potential coordinates
};

void bucket_release(Bucket& b) {
  if (b.stream) cudaStreamSynchronize(b.stream);
  if (b.graph) cudaGraphExecDestroy(b.graph);
  if (b.e64) {
    b.e64->release();
    delete b.e64;
  }
  if (b.e32) {
    b.e32->release();
    delete b.e32;
  }
  if (b.d64) cudaFree(b.d64);
  if (b.d32) cudaFree(b.d32);
  if (b.d_sc) cudaFree(b.d_sc);
  if (b.d_done) cudaFree(b.d_done);
  if (b.h_done) cudaFreeHost(b.h_done);
  if (b.stream) cudaStreamDestroy(b.stream);
  b = Bucket{};
}

// a bucket for requests of grid M (order N), with its plans (the planner's choice for that
// grid, as hom_create makes it), descriptor arrays and stream
int bucket_init(Bucket& b, const hom_request& r, const int* M, int cap) {
  b.d = r.d;
  b.nc = req_nc(r);
  for (int a = 0; a < 3; ++a) {
    b.M[a] = a < r.d ? M[a] : 1;
    b.N[a] = a < r.d ? r.N[a] : 1;
  }
  b.integration = r.integration;
  b.precision = r.precision;
  b.solver = r.solver;
  b.inner_form = r.opts.inner_form;
  b.cap = cap;
  b.slots.assign(b.cap, nullptr);
  b.nodes = 1;
  for (int a = 0; a < r.d; ++a) b.nodes *= M[a];
  b.red_grid = (int)std::min<long long>((b.nodes * b.nc + kThreads - 1) / kThreads, 152 * 8);
  int rc;
  if ((rc = alloc((void**)&b.d64, sizeof(ReqDesc<double>) * b.cap)) ||
      (rc = alloc((void**)&b.d32, sizeof(ReqDesc<float>) * b.cap)) ||
      (rc = alloc((void**)&b.d_sc, sizeof(Scalars*) * b.cap)) ||
      (rc = alloc((void**)&b.d_done, sizeof(int) * b.cap)))
    return rc;
  if (cudaMallocHost((void**)&b.h_done, sizeof(int) * b.cap) != cudaSuccess) {
    b.h_done = nullptr;
    return HOM_ERR_OOM;
  }
  if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess) {
    b.stream = nullptr;
    return HOM_ERR_CUDA;
  }
  const PlanChoice p64 = plan_choice(8, b.d, b.M, b.N, b.nc);
  b.e64 = new Engine<double>();
  if ((rc = b.e64->init(b.d, b.M, b.N, p64.budget, p64.rmax, p64.threads, p64.two_line, b.nc)))
    return rc;
  if (b.precision == HOM_FP32_REFINED) {
    const PlanChoice p32 = plan_choice(4, b.d, b.M, b.N, b.nc);
    b.e32 = new Engine<float>();
    if ((rc = b.e32->init(b.d, b.M, b.N, p32.budget, p32.rmax, p32.threads, p32.two_line, b.nc)))
      return rc;
  }
  return HOM_OK;
}

size_t estimate_bytes(const hom_request& r) {
  const int nc = req_nc(r);
  long long nodes = 1;
  for (int a = 0; a < r.d; ++a)
    nodes *= (r.integration == HOM_EXACT) ? (r.material.M[a] > 0 ? r.material.M[a] : 2 * r.N[a] - 1)
                                          : r.N[a];
  const long long nl = nodes / ((r.integration == HOM_EXACT)
                                    ? (r.material.M[r.d - 1] > 0 ? r.material.M[r.d - 1] : 2 * r.N[r.d - 1] - 1)
                                    : r.N[r.d - 1]);
  const int nlast = (int)(nodes / nl);
  size_t b = sizeof(double) * 5 * nc * nodes;                      // solver vectors
  b += sizeof(double) * 2 * nc * nl * ((nlast + 1) / 2);           // half spectrum
  b += nodes * 2 + sizeof(double) * nodes;                         // phases / coefficient field
  if (r.precision == HOM_FP32_REFINED) b += sizeof(float) * (4 * nc + 1) * nodes;
  const long long maxit = r.opts.fixed_iters > 0 ? r.opts.fixed_iters
                                                 : (r.opts.maxit > 0 ? r.opts.maxit : 100000);
  b += sizeof(double) * (size_t)std::min<long long>(maxit + 2, kHistMax);  // iteration history
  return b + (4u << 20);                                           // partials, plans, tables
}

}  // namespace

struct hom_server {
  size_t budget = 0, in_use = 0;
  int max_batch = 16;
  long long next_id = 1;
  std::deque<ServerReq*> queue;
  std::vector<Bucket> buckets;
  std::vector<hom_result> done;
  Scalars* d_idle = nullptr;
  int steps_per_graph = 4;
};

namespace {

int find_bucket(hom_server* S, const hom_request& r, const int* M) {
  for (size_t i = 0; i < S->buckets.size(); ++i) {
    const Bucket& b = S->buckets[i];
    bool same = b.d == r.d && b.nc == req_nc(r) && b.integration == r.integration &&
                b.precision == r.precision && b.solver == r.solver &&
                b.inner_form == r.opts.inner_form;
    for (int a = 0; a < r.d && same; ++a) same = b.M[a] == M[a] && b.N[a] == r.N[a];
    if (same) return (int)i;
  }
  return -1;
}

int bucket_upload(hom_server* S, Bucket& b) {
  std::vector<const Scalars*> scs(b.cap, nullptr);
  if (b.precision == HOM_FP32_REFINED) {
    std::vector<ReqDesc<float>> h(b.cap, idle_desc<float>(S->d_idle));
    for (int i = 0; i < b.cap; ++i)
      if (b.slots[i]) {
        h[i] = desc32(b.slots[i]->P);
        scs[i] = b.slots[i]->P->d_sc2;
      }
    HOM_CUDA(cudaMemcpyAsync(b.d32, h.data(), sizeof(ReqDesc<float>) * b.cap, cudaMemcpyHostToDevice, b.stream));
  } else {
    std::vector<ReqDesc<double>> h(b.cap, idle_desc<double>(S->d_idle));
    for (int i = 0; i < b.cap; ++i)
      if (b.slots[i]) {
        h[i] = desc64(b.slots[i]->P);
        scs[i] = b.slots[i]->P->d_sc;
      }
    HOM_CUDA(cudaMemcpyAsync(b.d64, h.data(), sizeof(ReqDesc<double>) * b.cap, cudaMemcpyHostToDevice, b.stream));
  }
  HOM_CUDA(cudaMemcpyAsync(b.d_sc, scs.data(), sizeof(Scalars*) * b.cap, cudaMemcpyHostToDevice, b.stream));
  HOM_CUDA(cudaStreamSynchronize(b.stream));  // host vectors go out of scope
  b.dirty = false;
  return HOM_OK;
}

void bucket_step(Bucket& b) {
  if (b.precision == HOM_FP32_REFINED)
    batch_step<float>(*b.e32, b.solver, b.d32, b.cap, b.red_grid, b.nodes, b.d, b.stream, b.pot);
  else
    batch_step<double>(*b.e64, b.solver, b.d64, b.cap, b.red_grid, b.nodes, b.d, b.stream);
}

int bucket_launch(hom_server* S, Bucket& b, int iterations) {
  if (!b.graph) {
    cudaGraph_t g = nullptr;
    const bool prof = profiling();
    if (prof) hom_profile_enable(0);
    HOM_CUDA(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
    const long long c0 = launch_counter();
    for (int k = 0; k < S->steps_per_graph; ++k) bucket_step(b);
    b.graph_launches = launch_counter() - c0;  // recorded, not run: counted per replay
    launch_counter() = c0;
    const cudaError_t e = cudaStreamEndCapture(b.stream, &g);
    if (prof) hom_profile_enable(1);
    HOM_CUDA(e);
    const cudaError_t e2 = cudaGraphInstantiate(&b.graph, g, 0);
    cudaGraphDestroy(g);
    HOM_CUDA(e2);
    b.graph_steps = S->steps_per_graph;
  }
  int k = 0;
  for (; k + b.graph_steps <= iterations; k += b.graph_steps) {
    HOM_CUDA(cudaGraphLaunch(b.graph, b.stream));
    launch_counter() += b.graph_launches;
  }
  for (; k < iterations; ++k) bucket_step(b);
  for (auto* r : b.slots)
    if (r) r->P->sv.issued += iterations;
  return check_last();
}

// a request that could not start: its result carries the status
void fail_request(hom_server* S, ServerReq* r, int status) {
  hom_result res{};
  res.id = r->id;
  res.status = status;
  res.latency_ms = ms_between(r->t_submit, Clock::now());
  S->done.push_back(res);
  delete r;
}

// move queued requests onto the device while the budget and the slots allow; each request's
// problem lives on its bucket's stream
int admit(hom_server* S) {
  while (!S->queue.empty()) {
    ServerReq* r = S->queue.front();
    if (S->in_use + r->bytes > S->budget && S->in_use > 0) break;
    int M[3];
    for (int a = 0; a < r->req.d; ++a)
      M[a] = (r->req.integration == HOM_EXACT)
                 ? (r->req.material.M[a] > 0 ? r->req.material.M[a] : 2 * r->req.N[a] - 1)
                 : r->req.N[a];
    int bi = find_bucket(S, r->req, M);
    if (bi >= 0) {
      Bucket& b = S->buckets[bi];
      if (std::find(b.slots.begin(), b.slots.end(), nullptr) == b.slots.end()) break;
    }
    S->queue.pop_front();
    int rc = HOM_OK;
    if (bi < 0) {
      Bucket nb;
      rc = bucket_init(nb, r->req, M, S->max_batch);
      if (rc != HOM_OK) {
        bucket_release(nb);
        fail_request(S, r, rc);
        continue;
      }
      S->buckets.push_back(nb);
      bi = (int)S->buckets.size() - 1;
    }
    Bucket& b = S->buckets[bi];
    // create the problem and start its session
    hom_material mat = r->req.material;
    mat.data = r->data.data();
    mat.table = r->table.empty() ? nullptr : r->table.data();
    mat.data_on_device = 0;
    hom_problem* P = nullptr;
    rc = hom_create(r->req.d, r->req.N, &mat, r->req.integration, r->req.precision, b.stream, &P);
    if (rc == HOM_OK)
      rc = hom_solve_begin(P, r->req.E, r->req.solver, r->req.tol, &r->req.opts);
    if (rc != HOM_OK) {
      if (P) hom_destroy(P);
      fail_request(S, r, rc);
      continue;
    }
    r->P = P;
    r->t_admit = Clock::now();
    S->in_use += r->bytes;
    b.pot = P->sv.pot;  // equal for every request of the bucket (same grid, solver, form)
    const int slot = (int)(std::find(b.slots.begin(), b.slots.end(), nullptr) - b.slots.begin());
    b.slots[slot] = r;
    r->bucket = bi;
    r->slot = slot;
    b.dirty = true;
  }
  return HOM_OK;
}

// finish a request whose solver stopped: outputs, timing, free its device memory
void retire(hom_server* S, Bucket& b, int slot) {
  ServerReq* r = b.slots[slot];
  hom_result res{};
  res.id = r->id;
  res.status = hom_solve_end(r->P, nullptr, &res.AH_EE, res.flux, &res.stats);
  const auto now = Clock::now();
  res.latency_ms = ms_between(r->t_submit, now);
  res.queue_ms = ms_between(r->t_submit, r->t_admit);
  S->done.push_back(res);
  hom_destroy(r->P);
  S->in_use -= r->bytes;
  b.slots[slot] = nullptr;
  b.dirty = true;
  delete r;
}

}  // namespace

extern "C" int hom_server_create(size_t hbm_budget_bytes, int max_batch, void* stream,
                                 hom_server** out) {
  if (!out || max_batch < 1 || hbm_budget_bytes == 0) return HOM_ERR_INVALID;
  (void)stream;  // every bucket runs on a stream of its own (see hom.h)
  auto* S = new hom_server();
  S->budget = hbm_budget_bytes;
  S->max_batch = max_batch;
  if (alloc((void**)&S->d_idle, sizeof(Scalars))) {
    delete S;
    return HOM_ERR_OOM;
  }
  Scalars idle{};
  idle.done = 1;
  cudaMemcpy(S->d_idle, &idle, sizeof(Scalars), cudaMemcpyHostToDevice);
  *out = S;
  return check_last();
}

extern "C" int hom_server_submit(hom_server* S, const hom_request* req, long long* id) {
  if (!S || !req || !id) return HOM_ERR_INVALID;
  if (req->d != 2 && req->d != 3) return HOM_ERR_INVALID;
  long long nodes = 1;
  for (int a = 0; a < req->d; ++a) {
    if (req->N[a] < 3 || req->N[a] % 2 == 0) return HOM_ERR_INVALID;
    nodes *= req->N[a];
  }
  auto* r = new ServerReq();
  r->req = *req;
  r->id = S->next_id++;
  r->t_submit = Clock::now();
  const hom_material& m = req->material;
  if (m.data_on_device || !m.data) {
    delete r;
    return HOM_ERR_INVALID;  // the server keeps host copies until admission
  }
  if (m.kind == HOM_A_PHASE || m.kind == HOM_A_STIFFNESS) {
    const int nc = req_nc(*req);
    if (!m.table || m.nphase < 1) {
      delete r;
      return HOM_ERR_INVALID;
    }
    r->data.assign((const unsigned char*)m.data, (const unsigned char*)m.data + nodes * m.index_bytes);
    r->table.assign(m.table, m.table + (size_t)m.nphase * nc * nc);
  } else if (m.kind == HOM_A_SCALAR) {
    r->data.assign((const unsigned char*)m.data, (const unsigned char*)m.data + nodes * sizeof(double));
  } else {
    long long mnodes = 1;
    for (int a = 0; a < req->d; ++a) mnodes *= (m.M[a] > 0 ? m.M[a] : 2 * req->N[a] - 1);
    r->data.assign((const unsigned char*)m.data, (const unsigned char*)m.data + mnodes * 2 * sizeof(double));
  }
  r->bytes = estimate_bytes(*req);
  S->queue.push_back(r);
  *id = r->id;
  return HOM_OK;
}

extern "C" int hom_server_step(hom_server* S, int iterations) {
  if (!S || iterations < 1) return HOM_ERR_INVALID;
  int rc = admit(S);
  if (rc) return rc;
  // one batched launch per pass and bucket, then the stopping flags of its slots in one copy.
  // Buckets without active slots are skipped entirely: their device descriptors may still
  // name the buffers of retired (freed) requests until the next upload.
  std::vector<char> live(S->buckets.size(), 0);
  for (size_t bi = 0; bi < S->buckets.size(); ++bi) {
    Bucket& b = S->buckets[bi];
    for (auto* r : b.slots) live[bi] = live[bi] || r != nullptr;
    if (!live[bi]) continue;
    if (b.dirty && (rc = bucket_upload(S, b))) return rc;
    if ((rc = bucket_launch(S, b, iterations))) return rc;
    k_gather_done<<<(b.cap + 127) / 128, 128, 0, b.stream>>>(b.d_sc, b.cap, b.d_done);
    HOM_CUDA(cudaMemcpyAsync(b.h_done, b.d_done, sizeof(int) * b.cap, cudaMemcpyDeviceToHost, b.stream));
  }
  // every live bucket's step is in flight on its own stream before the host waits for any
  for (size_t bi = 0; bi < S->buckets.size(); ++bi)
    if (live[bi]) HOM_CUDA(cudaStreamSynchronize(S->buckets[bi].stream));
  for (size_t bi = 0; bi < S->buckets.size(); ++bi) {
    if (!live[bi]) continue;
    Bucket& b = S->buckets[bi];
    for (int i = 0; i < b.cap; ++i) {
      ServerReq* r = b.slots[i];
      if (!r) continue;
      hom_problem* P = r->P;
      bool finished;
      if (P->sv.refined) {
        if (b.h_done[i] && !P->sv.finished) {
          if ((rc = refine_outer_update(P))) return rc;
        }
        finished = P->sv.finished;
      } else {
        const int cap = P->sv.maxit + (P->sv.solver == HOM_RICHARDSON ? 1 : 0);
        finished = b.h_done[i] || P->sv.issued >= cap;
      }
      if (finished) retire(S, b, i);
    }
  }
  return admit(S);
}

extern "C" int hom_server_poll(hom_server* S, hom_result* out, int max, int* count) {
  if (!S || !count || (max > 0 && !out)) return HOM_ERR_INVALID;
  const int n = std::min<int>(max, (int)S->done.size());
  for (int i = 0; i < n; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + n);
  *count = n;
  return HOM_OK;
}

extern "C" int hom_server_status(hom_server* S, int* active, int* queued, size_t* bytes_in_use) {
  if (!S) return HOM_ERR_INVALID;
  int a = 0;
  for (auto& b : S->buckets)
    for (auto* r : b.slots) a += r != nullptr;
  if (active) *active = a;
  if (queued) *queued = (int)S->queue.size();
  if (bytes_in_use) *bytes_in_use = S->in_use;
  return HOM_OK;
}

extern "C" void hom_server_destroy(hom_server* S) {
  if (!S) return;
  for (auto& b : S->buckets) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    for (auto* r : b.slots)
      if (r) {
        hom_destroy(r->P);
        delete r;
      }
    bucket_release(b);
  }
  for (auto* r : S->queue) delete r;
  cudaFree(S->d_idle);
  delete S;
}
