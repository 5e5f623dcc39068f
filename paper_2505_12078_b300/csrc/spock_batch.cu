// spock_batch.cu -- host side of the batched launch (include/spock.h,
// "batched solves"): problem descriptors packed on the device, the persistent
// k_batch launch with its prep and result kernels captured in a CUDA graph,
// and the warps-per-team autotuner.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/spock.h"
#include "spock_problem.h"

namespace spock {

cudaError_t launch_batch_f1(const Prob<float>*, const SolveBufs<float>*, const int*, const SolveOpts&,
                            const BatchPlan&, long long*, size_t, int, cudaStream_t);
cudaError_t launch_batch_d2(const Prob<double>*, const SolveBufs<double>*, const int*, const SolveOpts&,
                            const BatchPlan&, long long*, size_t, int, cudaStream_t);
int batch_grid_f1(size_t, int*);
int batch_grid_d2(size_t, int*);
size_t views_bytes_f1(int tw, int pipe_bytes);
size_t views_bytes_d2(int tw, int pipe_bytes);

namespace {

constexpr int kMaxWidth = 126;   // nx + nu of the batched kernels (D = 128 = nx + nu + 2)
// A problem whose evaluation of T moves more than kGangUnit bytes (factors and
// vector passes, iteration precision) is solved by a gang of CTAs, about one
// CTA per kGangUnit bytes (a power of two, at most kGangMax).
constexpr double kGangUnit = 4.0e6;
constexpr int kGangMax = 64;

template <class T>
struct BatchMeta {
  int n, n_nl, nx, nu;
  long long nv, o_x, o_u;
  const double* Sx;
  const double* SxN;
  const double* Su;
  T* x0s;
  SolveBufs<T> B;
  long long x0_off, x_off, u_off;
};

struct BatchOut {
  int status, iters, n_T, pad;
  double res_inf, risk;
  long long cycles;
};

// per problem (one CTA each): scaled x0, a zeroed control block, and a zero
// iterate unless warm-started
template <class T>
__global__ void k_batch_prep(const BatchMeta<T>* __restrict__ meta, int count, const double* __restrict__ x0,
                             int warm, int* __restrict__ next, unsigned* __restrict__ flags, int nflags) {
  const int p = blockIdx.x;
  if (p == 0 && threadIdx.x == 0) *next = 0;
  if (p == 0)
    for (int k = threadIdx.x; k < nflags; k += blockDim.x) flags[k] = 0u;
  if (p >= count) return;
  const BatchMeta<T> M = meta[p];
  for (int k = threadIdx.x; k < M.nx; k += blockDim.x) M.x0s[k] = (T)(M.Sx[k] * x0[M.x0_off + k]);
  int* c = reinterpret_cast<int*>(M.B.ctl);
  for (int k = threadIdx.x; k < (int)(sizeof(SolveCtl) / sizeof(int)); k += blockDim.x) c[k] = 0;
  if (!warm)
    for (long long e = threadIdx.x; e < M.nv; e += blockDim.x) M.B.V[e] = T(0);
}

// per problem (one CTA each): x = x~/S, u = u~/Su from T(v), the summary, and
// the final iterate moved into V for the next warm start
template <class T>
__global__ void k_batch_post(const BatchMeta<T>* __restrict__ meta, int count, double* __restrict__ xo,
                             double* __restrict__ uo, BatchOut* __restrict__ out,
                             const long long* __restrict__ cycles) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const BatchMeta<T> M = meta[p];
  const SolveCtl* c = M.B.ctl;
  const int fv = c->final_v, ftv = c->final_tv;
  T* bufs[4] = {M.B.V, M.B.TV, M.B.VT, M.B.TVT};
  const T* z = bufs[ftv & 3];
  const long long nX = (long long)M.n * M.nx, nU = (long long)M.n_nl * M.nu;
  if (xo)
    for (long long e = threadIdx.x; e < nX; e += blockDim.x) {
      const long long i = e / M.nx;
      const int k = (int)(e % M.nx);
      xo[M.x_off + e] = (double)z[M.o_x + e] / ((i >= M.n_nl) ? M.SxN[k] : M.Sx[k]);
    }
  if (uo)
    for (long long f = threadIdx.x; f < nU; f += blockDim.x) uo[M.u_off + f] = (double)z[M.o_u + f] / M.Su[f % M.nu];
  if (threadIdx.x == 0) {
    BatchOut o;
    o.status = c->status; o.iters = c->iters; o.n_T = c->n_T; o.pad = 0;
    o.res_inf = c->res_inf; o.risk = (double)z[0]; o.cycles = cycles ? cycles[p] : 0;
    out[p] = o;
  }
  __syncthreads();   // T(v) may sit in V: read it before v is moved there
  if ((fv & 3) != 0) {
    const T* v = bufs[fv & 3];
    for (long long e = threadIdx.x; e < M.nv; e += blockDim.x) M.B.V[e] = v[e];
  }
}

template <class T>
size_t views_bytes(int tw, int pipe_bytes) {
  return sizeof(T) == 8 ? views_bytes_d2(tw, pipe_bytes) : views_bytes_f1(tw, pipe_bytes);
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SPOCK_OK : SPOCK_EDEVICE; }

}  // namespace
}  // namespace spock

using namespace spock;

struct spock_batch {
  int count = 0, precision = 32;
  std::vector<spock_problem*> probs;
  std::vector<int> tw, pipe, order;     // per problem: warps per team, pipe bytes (0: off)
  std::vector<int> gang;                // per problem: CTAs of its gang (1: a single CTA)
  BatchPlan plan{};                     // device schedule (arrays below)
  int* d_plan = nullptr;                // gang_of | gang_start | gang_size | list_off | list | small_order
  unsigned* d_flags = nullptr;
  double* d_part = nullptr;
  std::vector<long long> x0_off, x_off, u_off;
  long long x0_total = 0, x_total = 0, u_total = 0;
  int optin = 0;
  DevMem mem;
  void* d_probs = nullptr;   // Prob<T>[count]
  void* d_bufs = nullptr;    // SolveBufs<T>[count]
  void* d_meta = nullptr;    // BatchMeta<T>[count]
  int *d_tw = nullptr, *d_next = nullptr;
  long long* d_cycles = nullptr;
  double *d_x0 = nullptr, *d_x = nullptr, *d_u = nullptr;
  BatchOut* d_out = nullptr;
  double *h_x0 = nullptr, *h_x = nullptr, *h_u = nullptr;
  BatchOut* h_out = nullptr;
  size_t smem = 0;
  int grid = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool have_graph = false;
  SolveOpts g_opts{};
  int g_warm = -1;
};

namespace {

template <class T>
Iter<T>& iter_of(spock_problem* p) {
  if constexpr (sizeof(T) == 8) return p->f64; else return p->f32;
}

// pipe bytes of the team sweeps for warps-per-team tw (0 when two buffers per
// team do not fit next to the views)
template <class T>
int team_pipe_bytes(const spock_problem* p, int tw, int optin) {
  const long long e = std::max((long long)p->nx * p->ldB,
                               (long long)(p->nx + p->nu) * p->ldF + (long long)p->nx * p->ldK);
  const int b = (int)(e * (long long)sizeof(T));
  const size_t need = views_bytes<T>(tw, b) + 16 * 1024;   // + static shared memory
  return need <= (size_t)optin ? b : 0;
}

int tw_min(const spock_problem* p) {
  const int d = p->nx + p->nu;
  int t = 1;
  while (64 * t < d) t *= 2;
  return t;
}

// bytes that one evaluation of T moves for problem p: the factors of both
// sweeps and about twenty vector passes
template <class T>
double t_bytes(const spock_problem* p) {
  const double f = (double)(p->n - 1) * ((double)p->nx * p->ldB + (double)(p->nx + p->nu) * p->ldF) +
                   (double)p->n_nl * ((double)p->nx * p->ldK + (double)p->nu * p->ldP);
  return (f + 20.0 * (double)p->nv) * sizeof(T);
}

// The gangs: each problem gets gang[p] = about one CTA per kGangUnit bytes of
// its T (a property of the problem alone, so a problem runs the same way in
// any batch). Problems with gang 1 go to the queue of single CTAs. For each
// larger gang size s, the class gets a number of gangs in proportion to its
// share of the batch's bytes (at least one); its problems are dealt to them
// largest first onto the least loaded gang. The rest of the grid serves the
// queue.
template <class T>
int build_plan(spock_batch* b) {
  const int n = b->count, grid = b->grid;
  b->gang.assign(n, 1);
  std::vector<double> w(n);
  double total = 0.0;
  for (int i = 0; i < n; ++i) {
    w[i] = t_bytes<T>(b->probs[i]);
    total += w[i];
    int s = 1;
    while (s < kGangMax && s * kGangUnit < w[i]) s *= 2;
    while (s > 1 && s > grid / 2) s /= 2;
    b->gang[i] = s;
  }
  std::vector<int> gang_of, gang_start, gang_size, list_off(1, 0), list, small;
  int used = 0;
  for (int s = kGangMax; s >= 2; s /= 2) {
    std::vector<int> cls;
    double cw = 0.0;
    for (int i : b->order)
      if (b->gang[i] == s) { cls.push_back(i); cw += w[i]; }
    if (cls.empty()) continue;
    int ng = (int)((cw / total) * grid / s);
    ng = std::max(1, std::min(ng, (int)cls.size()));
    while (ng > 1 && used + ng * s > grid - 1) --ng;
    if (used + ng * s > grid) {   // no room: the class joins the next smaller one
      for (int i : cls) b->gang[i] = s / 2;
      continue;
    }
    std::vector<double> load(ng, 0.0);
    std::vector<std::vector<int>> lists(ng);
    for (int i : cls) {
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[k].push_back(i);
      load[k] += w[i];
    }
    for (int k = 0; k < ng; ++k) {
      const int id = (int)gang_start.size();
      gang_start.push_back(used);
      gang_size.push_back(s);
      for (int c = 0; c < s; ++c) gang_of.push_back(id);
      used += s;
      list.insert(list.end(), lists[k].begin(), lists[k].end());
      list_off.push_back((int)list.size());
    }
  }
  for (int i : b->order)
    if (b->gang[i] == 1) small.push_back(i);
  // device copy: one int array
  std::vector<int> all;
  auto put = [&](const std::vector<int>& v) {
    const size_t o = all.size();
    all.insert(all.end(), v.begin(), v.end());
    return o;
  };
  const size_t o_of = put(gang_of), o_start = put(gang_start), o_size = put(gang_size), o_loff = put(list_off),
               o_list = put(list), o_small = put(small);
  if (b->d_plan) cudaFree(b->d_plan);
  b->d_plan = nullptr;
  if (cudaMalloc(&b->d_plan, sizeof(int) * std::max<size_t>(1, all.size())) != cudaSuccess) return SPOCK_ENOMEM;
  if (!all.empty() &&
      cudaMemcpy(b->d_plan, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return SPOCK_EDEVICE;
  BatchPlan& P = b->plan;
  P.n_gang_ctas = used;
  P.gang_of = b->d_plan + o_of;
  P.gang_start = b->d_plan + o_start;
  P.gang_size = b->d_plan + o_size;
  P.list_off = b->d_plan + o_loff;
  P.list = b->d_plan + o_list;
  P.small_order = b->d_plan + o_small;
  P.n_small = (int)small.size();
  P.next = b->d_next;
  P.flags = b->d_flags;
  P.partials = b->d_part;
  return SPOCK_OK;
}

// descriptors of every problem with the current tw / pipe choice, and the
// launch's shared memory, grid and plan
template <class T>
int upload_desc(spock_batch* b) {
  std::vector<Prob<T>> P(b->count);
  size_t smem = 0;
  for (int i = 0; i < b->count; ++i) {
    P[i] = iter_of<T>(b->probs[i]).P;
    P[i].cta = 0;
    P[i].pipe_bytes = b->pipe[i];
    smem = std::max(smem, views_bytes<T>(b->tw[i], b->pipe[i]));
  }
  if (cudaMemcpy(b->d_probs, P.data(), sizeof(Prob<T>) * b->count, cudaMemcpyHostToDevice) != cudaSuccess)
    return SPOCK_EDEVICE;
  if (cudaMemcpy(b->d_tw, b->tw.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice) != cudaSuccess)
    return SPOCK_EDEVICE;
  b->smem = smem;
  int g = 0;
  const int rc = sizeof(T) == 8 ? batch_grid_d2(smem, &g) : batch_grid_f1(smem, &g);
  if (rc || g <= 0) return SPOCK_EDEVICE;
  b->grid = g;
  if (b->have_graph) {
    cudaGraphExecDestroy(b->exec);
    b->have_graph = false;
  }
  return build_plan<T>(b);
}

template <class T>
int batch_init(spock_batch* b) {
  const int n = b->count;
  std::vector<SolveBufs<T>> B(n);
  std::vector<BatchMeta<T>> M(n);
  for (int i = 0; i < n; ++i) {
    spock_problem* p = b->probs[i];
    Iter<T>& it = iter_of<T>(p);
    const int rc = ensure_bufs<T>(p, it);
    if (rc) return rc;
    B[i] = it.sb;
    BatchMeta<T>& m = M[i];
    m.n = p->n; m.n_nl = p->n_nl; m.nx = p->nx; m.nu = p->nu;
    m.nv = p->nv; m.o_x = p->o_x; m.o_u = p->o_u;
    m.Sx = p->d_Sx; m.SxN = p->d_SxN; m.Su = p->d_Su;
    m.x0s = it.x0s;
    m.B = it.sb;
    m.x0_off = b->x0_off[i]; m.x_off = b->x_off[i]; m.u_off = b->u_off[i];
  }
  DevMem& m = b->mem;
  b->d_probs = m.alloc<Prob<T>>(n);
  b->d_bufs = m.alloc<SolveBufs<T>>(n);
  b->d_meta = m.alloc<BatchMeta<T>>(n);
  if (m.failed) return SPOCK_ENOMEM;
  if (cudaMemcpy(b->d_bufs, B.data(), sizeof(SolveBufs<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_meta, M.data(), sizeof(BatchMeta<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return SPOCK_EDEVICE;
  return upload_desc<T>(b);
}

template <class T>
cudaError_t enqueue(spock_batch* b, const SolveOpts& so, int warm, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(b->d_x0, b->h_x0, sizeof(double) * b->x0_total, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  k_batch_prep<T><<<b->count, 256, 0, st>>>((const BatchMeta<T>*)b->d_meta, b->count, b->d_x0, warm, b->d_next,
                                            b->d_flags, b->plan.n_gang_ctas);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if constexpr (sizeof(T) == 8)
    e = launch_batch_d2((const Prob<double>*)b->d_probs, (const SolveBufs<double>*)b->d_bufs, b->d_tw, so, b->plan,
                        b->d_cycles, b->smem, b->grid, st);
  else
    e = launch_batch_f1((const Prob<float>*)b->d_probs, (const SolveBufs<float>*)b->d_bufs, b->d_tw, so, b->plan,
                        b->d_cycles, b->smem, b->grid, st);
  if (e != cudaSuccess) return e;
  k_batch_post<T><<<b->count, 256, 0, st>>>((const BatchMeta<T>*)b->d_meta, b->count, b->d_x, b->d_u, b->d_out,
                                            b->d_cycles);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaMemcpyAsync(b->h_out, b->d_out, sizeof(BatchOut) * b->count, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(b->h_x, b->d_x, sizeof(double) * b->x_total, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(b->h_u, b->d_u, sizeof(double) * b->u_total, cudaMemcpyDeviceToHost, st);
}

bool same_opts(const SolveOpts& a, const SolveOpts& b) {
  return a.tol == b.tol && a.max_iters == b.max_iters && a.max_backtracks == b.max_backtracks &&
         a.method == b.method && a.rank_tol == b.rank_tol && a.aa_qr == b.aa_qr;
}

// one replay of the captured graph (captured anew when the options change)
template <class T>
int run_graph(spock_batch* b, const SolveOpts& so, int warm, float* ms) {
  if (!b->have_graph || !same_opts(so, b->g_opts) || warm != b->g_warm) {
    if (b->have_graph) {
      cudaGraphExecDestroy(b->exec);
      b->have_graph = false;
    }
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPOCK_EDEVICE;
    const cudaError_t e = enqueue<T>(b, so, warm, b->stream);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) return SPOCK_EDEVICE;
    const cudaError_t e3 = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) return SPOCK_EDEVICE;
    b->have_graph = true;
    b->g_opts = so;
    b->g_warm = warm;
  }
  cudaEventRecord(b->e0, b->stream);
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return SPOCK_EDEVICE;
  cudaEventRecord(b->e1, b->stream);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SPOCK_EDEVICE;
  if (ms) cudaEventElapsedTime(ms, b->e0, b->e1);
  return SPOCK_OK;
}

void order_by_work(spock_batch* b) {
  std::vector<double> w(b->count);
  for (int i = 0; i < b->count; ++i) {
    const spock_problem* p = b->probs[i];
    w[i] = (double)p->n * (p->nx + p->nu) * (p->nx + p->nu);
  }
  b->order.resize(b->count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return w[a] > w[c]; });
}

void default_choice(spock_batch* b) {
  b->tw.resize(b->count);
  b->pipe.resize(b->count);
  for (int i = 0; i < b->count; ++i) {
    b->tw[i] = tw_min(b->probs[i]);
    b->pipe[i] = (b->precision == 64) ? team_pipe_bytes<double>(b->probs[i], b->tw[i], b->optin)
                                      : team_pipe_bytes<float>(b->probs[i], b->tw[i], b->optin);
  }
}

int clock_khz() {
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  return khz > 0 ? khz : 1;
}

}  // namespace

extern "C" {

int spock_batch_create(spock_problem* const* problems, int count, int precision, spock_batch** out) {
  if (!out) return SPOCK_EINVAL;
  *out = nullptr;
  if (!problems || count < 1 || (precision != 32 && precision != 64)) return SPOCK_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!problems[i]) return SPOCK_EINVAL;
    if (problems[i]->nx + problems[i]->nu > kMaxWidth) return SPOCK_EUNSUPPORTED;
    if (problems[i]->l1 > 0 || problems[i]->tv || problems[i]->soft) return SPOCK_EUNSUPPORTED;   // single-problem calls only
  }
  spock_batch* b = new spock_batch();
  b->count = count;
  b->precision = precision;
  b->probs.assign(problems, problems + count);
  b->x0_off.resize(count); b->x_off.resize(count); b->u_off.resize(count);
  for (int i = 0; i < count; ++i) {
    const spock_problem* p = problems[i];
    b->x0_off[i] = b->x0_total; b->x_off[i] = b->x_total; b->u_off[i] = b->u_total;
    b->x0_total += p->nx;
    b->x_total += (long long)p->n * p->nx;
    b->u_total += (long long)p->n_nl * p->nu;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  order_by_work(b);
  default_choice(b);
  DevMem& m = b->mem;
  b->d_tw = m.alloc<int>(count);
  b->d_next = m.alloc<int>(1);
  b->d_cycles = m.alloc<long long>(count);
  b->d_x0 = m.alloc<double>(b->x0_total);
  b->d_x = m.alloc<double>(b->x_total);
  b->d_u = m.alloc<double>(b->u_total);
  b->d_out = m.alloc<BatchOut>(count);
  {
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->d_flags = m.alloc<unsigned>((long long)nsm * 8);
    b->d_part = m.alloc<double>((long long)2 * NRED * nsm * 8);
  }
  if (m.failed) { m.free_all(); delete b; return SPOCK_ENOMEM; }
  if (cudaMallocHost(&b->h_x0, sizeof(double) * b->x0_total) != cudaSuccess ||
      cudaMallocHost(&b->h_x, sizeof(double) * b->x_total) != cudaSuccess ||
      cudaMallocHost(&b->h_u, sizeof(double) * b->u_total) != cudaSuccess ||
      cudaMallocHost(&b->h_out, sizeof(BatchOut) * count) != cudaSuccess) {
    spock_batch_destroy(b);
    return SPOCK_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) {
    spock_batch_destroy(b);
    return SPOCK_EDEVICE;
  }
  cudaMemset(b->d_cycles, 0, sizeof(long long) * count);
  const int rc = precision == 64 ? batch_init<double>(b) : batch_init<float>(b);
  if (rc) { spock_batch_destroy(b); return rc; }
  *out = b;
  return cuda_rc(cudaDeviceSynchronize());
}

void spock_batch_destroy(spock_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->have_graph) cudaGraphExecDestroy(b->exec);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->h_x0) cudaFreeHost(b->h_x0);
  if (b->h_x) cudaFreeHost(b->h_x);
  if (b->h_u) cudaFreeHost(b->h_u);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->d_plan) cudaFree(b->d_plan);
  b->mem.free_all();
  delete b;
}

int spock_batch_sizes(const spock_batch* b, long long* x0_total, long long* x_total, long long* u_total) {
  if (!b) return SPOCK_EINVAL;
  if (x0_total) *x0_total = b->x0_total;
  if (x_total) *x_total = b->x_total;
  if (u_total) *u_total = b->u_total;
  return SPOCK_OK;
}

int spock_batch_set_tw(spock_batch* b, const int* tw) {
  if (!b) return SPOCK_EINVAL;
  if (!tw) {
    default_choice(b);
  } else {
    for (int i = 0; i < b->count; ++i)
      if (!(tw[i] == 1 || tw[i] == 2 || tw[i] == 4 || tw[i] == 8) || tw[i] < tw_min(b->probs[i]))
        return SPOCK_EINVAL;
    for (int i = 0; i < b->count; ++i) {
      b->tw[i] = tw[i];
      b->pipe[i] = (b->precision == 64) ? team_pipe_bytes<double>(b->probs[i], tw[i], b->optin)
                                        : team_pipe_bytes<float>(b->probs[i], tw[i], b->optin);
    }
  }
  return b->precision == 64 ? upload_desc<double>(b) : upload_desc<float>(b);
}

int spock_batch_autotune(spock_batch* b, int iters, int* tw_out) {
  if (!b || iters < 1) return SPOCK_EINVAL;
  const int n = b->count;
  std::vector<long long> best(n, -1);
  std::vector<int> best_tw(b->tw), best_pipe(b->pipe);
  SolveOpts so{};
  so.tol = 0.0; so.max_iters = iters; so.max_backtracks = 1; so.method = 1;
  so.rank_tol = b->precision == 64 ? 1e-10 : 1e-5;
  memset(b->h_x0, 0, sizeof(double) * b->x0_total);
  std::vector<long long> cyc(n);
  for (int t : {1, 2, 4, 8}) {
    for (int pipe_on = 0; pipe_on < 2; ++pipe_on) {
      bool any = false;
      for (int i = 0; i < n; ++i) {
        const int tw = std::max(t, tw_min(b->probs[i]));
        b->tw[i] = tw;
        const int pb = (b->precision == 64) ? team_pipe_bytes<double>(b->probs[i], tw, b->optin)
                                            : team_pipe_bytes<float>(b->probs[i], tw, b->optin);
        b->pipe[i] = pipe_on ? pb : 0;
        any = any || (tw == t && (pipe_on == 0 || pb > 0));
      }
      if (!any) continue;
      int rc = b->precision == 64 ? upload_desc<double>(b) : upload_desc<float>(b);
      if (rc) return rc;
      rc = b->precision == 64 ? run_graph<double>(b, so, 0, nullptr) : run_graph<float>(b, so, 0, nullptr);
      if (rc) return rc;
      for (int i = 0; i < n; ++i) {
        const long long c = b->h_out[i].cycles;
        if (b->h_out[i].status < 0) continue;
        if (best[i] < 0 || c < best[i]) {
          best[i] = c;
          best_tw[i] = b->tw[i];
          best_pipe[i] = b->pipe[i];
        }
      }
    }
  }
  b->tw = best_tw;
  b->pipe = best_pipe;
  if (tw_out)
    for (int i = 0; i < n; ++i) tw_out[i] = b->tw[i];
  // leave every iterate at zero
  int rc = b->precision == 64 ? upload_desc<double>(b) : upload_desc<float>(b);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    spock_problem* p = b->probs[i];
    if (b->precision == 64) cudaMemset(p->f64.sb.V, 0, p->nv * 8);
    else cudaMemset(p->f32.sb.V, 0, p->nv * 4);
  }
  return cuda_rc(cudaDeviceSynchronize());
}

int spock_batch_solve(spock_batch* b, const double* x0, const spock_solve_opts* opts, double* x_out,
                      double* u_out, double* risk, spock_batch_info* info, double* total_ms) {
  if (!b || !x0) return SPOCK_EINVAL;
  spock_solve_opts o;
  if (opts) o = *opts;
  else { spock_solve_opts_default(&o); o.precision = b->precision; }
  if (o.precision != b->precision || !(o.tol >= 0) || o.max_iters < 0 || o.max_backtracks < 1 ||
      o.method < 0 || o.method > 1)
    return SPOCK_EINVAL;
  for (long long k = 0; k < b->x0_total; ++k)
    if (!isfinite(x0[k])) return SPOCK_EINVAL;
  memcpy(b->h_x0, x0, sizeof(double) * b->x0_total);
  SolveOpts so{};
  so.tol = o.tol; so.max_iters = o.max_iters; so.max_backtracks = o.max_backtracks; so.method = o.method;
  so.rank_tol = (o.precision == 64) ? 1e-10 : 1e-5;
  so.aa_qr = o.aa_mode == 1 ? 1 : 0;
  float ms = 0.f;
  const int rc = b->precision == 64 ? run_graph<double>(b, so, o.warm_start ? 1 : 0, &ms)
                                    : run_graph<float>(b, so, o.warm_start ? 1 : 0, &ms);
  if (rc) return rc;
  if (total_ms) *total_ms = ms;
  if (x_out) memcpy(x_out, b->h_x, sizeof(double) * b->x_total);
  if (u_out) memcpy(u_out, b->h_u, sizeof(double) * b->u_total);
  const double khz = (double)clock_khz();
  int worst = SPOCK_OK;
  for (int i = 0; i < b->count; ++i) {
    const BatchOut& r = b->h_out[i];
    const int st = r.status == 0 ? SPOCK_OK : (r.status > 0 ? SPOCK_MAXITER : SPOCK_ETIMEOUT);
    if (st < 0 && worst >= 0) worst = st;
    else if (st == SPOCK_MAXITER && worst == SPOCK_OK) worst = st;
    if (risk) risk[i] = r.risk;
    if (info) {
      info[i].status = st;
      info[i].iters = r.iters;
      info[i].n_T = r.n_T;
      info[i].tw = b->tw[i];
      info[i].res_inf = r.res_inf;
      info[i].risk = r.risk;
      info[i].device_ms = (double)r.cycles / khz;
      info[i].xi1 = info[i].xi2 = info[i].infeas = info[i].gap = NAN;
    }
  }
  if (info && o.fp64_check) {
    // FP64 exit check of every final iterate (kept in V by k_batch_post)
    for (int i = 0; i < b->count; ++i) {
      spock_problem* p = b->probs[i];
      double o7[7];
      const void* v = b->precision == 64 ? (const void*)p->f64.sb.V : (const void*)p->f32.sb.V;
      const int rc2 = check_fp64(p, b->precision, v, b->stream, o7);
      if (rc2) return rc2;
      info[i].xi1 = o7[1]; info[i].xi2 = o7[2]; info[i].infeas = o7[3]; info[i].gap = o7[4];
    }
  }
  return worst;
}

}  // extern "C"
