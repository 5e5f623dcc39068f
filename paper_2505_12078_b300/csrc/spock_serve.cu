// spock_serve.cu -- host side of serving (include/spock.h, "serving"):
// resident plants (problems with their factors and warm-start iterates on the
// device), admission by device memory, a request ring in mapped host memory
// drained by the persistent k_serve launch, and per-plant ordering of requests.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <vector>

#include "../../include/spock.h"
#include "spock_problem.h"

namespace spock {

cudaError_t launch_serve_f1(const Prob<float>*, const SolveBufs<float>*, const int*, const ServeMeta<float>*,
                            const SolveOpts&, const ServeReq*, ServeRes*, int, ServeCtl*, ServeDev*,
                            unsigned long long, size_t, int, cudaStream_t);
cudaError_t launch_serve_d2(const Prob<double>*, const SolveBufs<double>*, const int*, const ServeMeta<double>*,
                            const SolveOpts&, const ServeReq*, ServeRes*, int, ServeCtl*, ServeDev*,
                            unsigned long long, size_t, int, cudaStream_t);
int serve_grid_f1(size_t, int*);
int serve_grid_d2(size_t, int*);
size_t views_bytes_f1(int tw, int pipe_bytes);
size_t views_bytes_d2(int tw, int pipe_bytes);

}  // namespace spock

using namespace spock;

namespace {

using Clock = std::chrono::steady_clock;
constexpr unsigned long long kIdleNs = 1000000000ull;   // k_serve leaves after 1 s without requests

struct Pending {
  long long id;
  int warm;
  double x0[SERVE_MAX_NX];
  Clock::time_point t_submit;
};

}  // namespace

struct spock_server {
  int count = 0, precision = 32, admitted = 0, cap = 0;
  std::vector<spock_problem*> plants;
  std::vector<int> is_admitted;     // per plant: its solve buffers are resident for the server
  std::vector<long long> charged;   // per plant: bytes charged to the budget at admission
  std::vector<int> release_pending; // per plant: evicted, buffers freed once the launch is idle
  long long budget = 0;             // explicit admission budget (0: free device memory)
  long long room = 0;               // budget left (explicit budget only)
  SolveOpts so{};
  DevMem mem;
  void *d_probs = nullptr, *d_bufs = nullptr, *d_meta = nullptr;
  int* d_tw = nullptr;
  ServeDev* d_dev = nullptr;
  ServeReq *h_ring = nullptr, *d_ring = nullptr;
  ServeRes *h_res = nullptr, *d_res = nullptr;
  ServeCtl *h_ctl = nullptr, *d_ctl = nullptr;
  size_t smem = 0;
  int grid = 0;
  cudaStream_t stream = nullptr;
  bool launched = false;
  long long tail = 0, next_id = 0;
  std::vector<int> slot_busy;                      // ring slot holds an unfinished request
  std::vector<int> slot_plant;
  std::vector<Clock::time_point> slot_submit;
  std::vector<int> plant_busy;                     // a request of the plant is on the device
  std::vector<std::deque<Pending>> queue;          // per plant, waiting for the plant
  long long outstanding = 0;
};

namespace {

template <class T>
Iter<T>& iter_of(spock_problem* p) {
  if constexpr (sizeof(T) == 8) return p->f64; else return p->f32;
}

int tw_min(const spock_problem* p) {
  const int d = p->nx + p->nu;
  int t = 1;
  while (64 * t < d) t *= 2;
  return t;
}

template <class T>
size_t views_bytes(int tw, int pipe_bytes) {
  return sizeof(T) == 8 ? views_bytes_d2(tw, pipe_bytes) : views_bytes_f1(tw, pipe_bytes);
}

// device memory kept free for the launch, the ring and other users
constexpr long long kReserve = 256ll << 20;

long long free_room() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
  return (long long)fr - kReserve;
}

template <class T>
int serve_init(spock_server* s) {
  const int n = s->count;
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  std::vector<Prob<T>> P(n);
  std::vector<SolveBufs<T>> B(n);
  std::vector<ServeMeta<T>> M(n);
  std::vector<int> tw(n);
  size_t smem = 0;
  // descriptors, team widths and shared memory of every plant (admitted now or
  // later): they depend on the plant's sizes only
  for (int i = 0; i < n; ++i) {
    spock_problem* p = s->plants[i];
    Iter<T>& it = iter_of<T>(p);
    tw[i] = tw_min(p);
    const long long e = std::max((long long)p->nx * p->ldB,
                                 (long long)(p->nx + p->nu) * p->ldF + (long long)p->nx * p->ldK);
    const int pb = (int)(e * (long long)sizeof(T));
    P[i] = it.P;
    P[i].cta = 0;
    P[i].pipe_bytes = (views_bytes<T>(tw[i], pb) + 16 * 1024 <= (size_t)optin) ? pb : 0;
    smem = std::max(smem, views_bytes<T>(tw[i], P[i].pipe_bytes));
    if (s->is_admitted[i]) {
      const int rc = ensure_bufs<T>(p, it);
      if (rc) return rc;
      B[i] = it.sb;
    }
    M[i].nx = p->nx; M[i].nu = p->nu; M[i].o_u = p->o_u; M[i].nv = p->nv;
    M[i].Sx = p->d_Sx; M[i].Su = p->d_Su; M[i].x0s = it.x0s;
  }
  DevMem& m = s->mem;
  s->d_probs = m.alloc<Prob<T>>(n);
  s->d_bufs = m.alloc<SolveBufs<T>>(n);
  s->d_meta = m.alloc<ServeMeta<T>>(n);
  s->d_tw = m.alloc<int>(n);
  s->d_dev = m.alloc<ServeDev>(1);
  if (m.failed) return SPOCK_ENOMEM;
  if (cudaMemcpy(s->d_probs, P.data(), sizeof(Prob<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_bufs, B.data(), sizeof(SolveBufs<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_meta, M.data(), sizeof(ServeMeta<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_tw, tw.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->d_dev, 0, sizeof(ServeDev)) != cudaSuccess)
    return SPOCK_EDEVICE;
  s->smem = smem;
  int g = 0;
  const int rc = sizeof(T) == 8 ? serve_grid_d2(smem, &g) : serve_grid_f1(smem, &g);
  if (rc || g <= 0) return SPOCK_EDEVICE;
  s->grid = g;
  return SPOCK_OK;
}

// bytes admission charges for plant i: its solve buffers, unless they exist
long long admission_need(const spock_server* s, int i) {
  const spock_problem* p = s->plants[i];
  const bool have = s->precision == 64 ? p->f64.have_bufs : p->f32.have_bufs;
  return have ? 0 : solve_buffer_bytes(p, s->precision);
}

// room for a new admission: the explicit budget left, never more than the
// free device memory less the reserve
long long admission_room(const spock_server* s) {
  const long long fr = free_room();
  return s->budget > 0 ? std::min(s->room, fr) : fr;
}

// free the buffers of evicted plants once no launch can touch them
void release_evicted(spock_server* s, bool force) {
  if (!force && s->launched && cudaStreamQuery(s->stream) != cudaSuccess) return;
  for (int i = 0; i < s->count; ++i) {
    if (!s->release_pending[i]) continue;
    if (s->precision == 64) release_bufs(s->plants[i]->f64);
    else release_bufs(s->plants[i]->f32);
    s->release_pending[i] = 0;
  }
}

// admit plant i now (a request for it arrived): allocate its buffers if the
// room allows and publish its table entry before any request can name it
template <class T>
int admit_plant(spock_server* s, int i) {
  spock_problem* p = s->plants[i];
  Iter<T>& it = iter_of<T>(p);
  // evicted with buffers not freed yet: taking them back costs their bytes
  const long long need = s->release_pending[i] ? solve_buffer_bytes(p, s->precision) : admission_need(s, i);
  if (need > admission_room(s)) return SPOCK_ENOMEM;
  s->release_pending[i] = 0;
  const int rc = ensure_bufs<T>(p, it);
  if (rc) return rc;
  // the persistent launch may be running: the entry is written with a
  // synchronous copy before the host publishes any request of plant i, and
  // k_serve reads entries through L2 (never a stale non-coherent line)
  if (cudaMemcpy(static_cast<SolveBufs<T>*>(s->d_bufs) + i, &it.sb, sizeof(SolveBufs<T>), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return SPOCK_EDEVICE;
  s->is_admitted[i] = 1;
  s->charged[i] = need;
  if (s->budget > 0) s->room -= need;
  s->admitted += 1;
  return SPOCK_OK;
}

template <class T>
cudaError_t relaunch(spock_server* s) {
  if constexpr (sizeof(T) == 8)
    return launch_serve_d2((const Prob<double>*)s->d_probs, (const SolveBufs<double>*)s->d_bufs, s->d_tw,
                           (const ServeMeta<double>*)s->d_meta, s->so, s->d_ring, s->d_res, s->cap, s->d_ctl,
                           s->d_dev, kIdleNs, s->smem, s->grid, s->stream);
  else
    return launch_serve_f1((const Prob<float>*)s->d_probs, (const SolveBufs<float>*)s->d_bufs, s->d_tw,
                           (const ServeMeta<float>*)s->d_meta, s->so, s->d_ring, s->d_res, s->cap, s->d_ctl,
                           s->d_dev, kIdleNs, s->smem, s->grid, s->stream);
}

// the persistent launch is running, or started (it leaves after kIdleNs idle)
int ensure_running(spock_server* s) {
  if (s->launched && cudaStreamQuery(s->stream) == cudaErrorNotReady) return SPOCK_OK;
  if (s->launched && cudaStreamQuery(s->stream) != cudaSuccess) return SPOCK_EDEVICE;
  const cudaError_t e = s->precision == 64 ? relaunch<double>(s) : relaunch<float>(s);
  if (e != cudaSuccess) return SPOCK_EDEVICE;
  s->launched = true;
  return SPOCK_OK;
}

// publish request r of plant p into the next ring slot (false: slot busy)
bool publish(spock_server* s, int p, const Pending& r) {
  const int slot = (int)(s->tail % s->cap);
  if (s->slot_busy[slot]) return false;
  ServeReq& q = s->h_ring[slot];
  q.plant = p;
  q.warm = r.warm;
  q.id = r.id;
  memcpy(q.x0, r.x0, sizeof(q.x0));
  s->h_res[slot].done = 0;
  s->slot_busy[slot] = 1;
  s->slot_plant[slot] = p;
  s->slot_submit[slot] = r.t_submit;
  s->plant_busy[p] = 1;
  std::atomic_thread_fence(std::memory_order_release);
  s->tail += 1;
  s->h_ctl->tail = s->tail;
  return true;
}

}  // namespace

extern "C" {

int spock_server_create(spock_problem* const* plants, int count, int precision, const spock_solve_opts* opts,
                        int ring_slots, long long mem_budget, spock_server** out, int* admitted) {
  if (!out) return SPOCK_EINVAL;
  *out = nullptr;
  if (!plants || count < 1 || (precision != 32 && precision != 64) || ring_slots < 1) return SPOCK_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!plants[i]) return SPOCK_EINVAL;
    if (plants[i]->nx > SERVE_MAX_NX || plants[i]->nu > SERVE_MAX_NU || plants[i]->nx + plants[i]->nu > 126)
      return SPOCK_EUNSUPPORTED;
    if (plants[i]->l1 > 0 || plants[i]->tv || plants[i]->soft) return SPOCK_EUNSUPPORTED;   // single-problem calls only
  }
  spock_solve_opts o;
  if (opts) o = *opts;
  else { spock_solve_opts_default(&o); o.precision = precision; }
  if (o.precision != precision || !(o.tol >= 0) || o.max_iters < 0 || o.max_backtracks < 1 || o.method < 0 ||
      o.method > 1)
    return SPOCK_EINVAL;
  spock_server* s = new spock_server();
  s->count = count;
  s->precision = precision;
  s->plants.assign(plants, plants + count);
  s->so.tol = o.tol; s->so.max_iters = o.max_iters; s->so.max_backtracks = o.max_backtracks;
  s->so.method = o.method; s->so.rank_tol = precision == 64 ? 1e-10 : 1e-5;
  s->so.aa_qr = o.aa_mode == 1 ? 1 : 0;
  // admission by device memory: plants in order while their solve buffers fit
  // in the budget (an explicit budget is clamped to the free memory less the
  // reserve; by default the free memory less the reserve)
  s->is_admitted.assign(count, 0);
  s->charged.assign(count, 0);
  s->release_pending.assign(count, 0);
  const long long fr = free_room();
  s->budget = mem_budget > 0 ? mem_budget : 0;
  long long room = mem_budget > 0 ? std::min((long long)mem_budget, fr) : fr;
  int adm = 0;
  for (int i = 0; i < count; ++i) {
    const long long need = admission_need(s, i);
    if (need > room) break;
    room -= need;
    s->is_admitted[i] = 1;
    s->charged[i] = need;
    ++adm;
  }
  s->room = mem_budget > 0 ? room : 0;
  s->admitted = adm;
  if (admitted) *admitted = adm;
  if (adm == 0) { delete s; return SPOCK_ENOMEM; }
  s->cap = ring_slots;
  s->slot_busy.assign(ring_slots, 0);
  s->slot_plant.assign(ring_slots, -1);
  s->slot_submit.resize(ring_slots);
  s->plant_busy.assign(count, 0);
  s->queue.resize(count);
  if (cudaHostAlloc(&s->h_ring, sizeof(ServeReq) * ring_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->h_res, sizeof(ServeRes) * ring_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->h_ctl, sizeof(ServeCtl), cudaHostAllocMapped) != cudaSuccess) {
    spock_server_destroy(s);
    return SPOCK_ENOMEM;
  }
  memset(s->h_ring, 0, sizeof(ServeReq) * ring_slots);
  memset(s->h_res, 0, sizeof(ServeRes) * ring_slots);
  memset((void*)s->h_ctl, 0, sizeof(ServeCtl));
  cudaHostGetDevicePointer((void**)&s->d_ring, s->h_ring, 0);
  cudaHostGetDevicePointer((void**)&s->d_res, s->h_res, 0);
  cudaHostGetDevicePointer((void**)&s->d_ctl, (void*)s->h_ctl, 0);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    spock_server_destroy(s);
    return SPOCK_EDEVICE;
  }
  const int rc = precision == 64 ? serve_init<double>(s) : serve_init<float>(s);
  if (rc) { spock_server_destroy(s); return rc; }
  if (cudaDeviceSynchronize() != cudaSuccess) { spock_server_destroy(s); return SPOCK_EDEVICE; }
  *out = s;
  return adm == count ? SPOCK_OK : SPOCK_PARTIAL;
}

int spock_server_submit(spock_server* s, int plant, const double* x0, int warm_start, long long* id_out) {
  if (!s || !x0 || plant < 0 || plant >= s->count) return SPOCK_EINVAL;
  const int nx = s->plants[plant]->nx;
  for (int k = 0; k < nx; ++k)
    if (!isfinite(x0[k])) return SPOCK_EINVAL;
  if (!s->is_admitted[plant]) {           // refused or evicted earlier: try again now
    release_evicted(s, false);
    const int rc = s->precision == 64 ? admit_plant<double>(s, plant) : admit_plant<float>(s, plant);
    if (rc) return rc;
  }
  Pending r;
  r.id = s->next_id++;
  r.warm = warm_start ? 1 : 0;
  memset(r.x0, 0, sizeof(r.x0));
  memcpy(r.x0, x0, sizeof(double) * nx);
  r.t_submit = Clock::now();
  if (id_out) *id_out = r.id;
  s->outstanding += 1;
  if (s->plant_busy[plant] || !s->queue[plant].empty() || !publish(s, plant, r)) {
    s->queue[plant].push_back(r);
    return SPOCK_OK;
  }
  return ensure_running(s);
}

int spock_server_poll(spock_server* s, spock_serve_result* out, int max_out, int* n_out) {
  if (!s || (max_out > 0 && !out)) return SPOCK_EINVAL;
  int n = 0;
  for (int slot = 0; slot < s->cap && n < max_out; ++slot) {
    if (!s->slot_busy[slot] || !s->h_res[slot].done) continue;
    std::atomic_thread_fence(std::memory_order_acquire);
    const ServeRes& r = s->h_res[slot];
    const int p = s->slot_plant[slot];
    spock_serve_result& o = out[n++];
    o.id = r.id;
    o.plant = p;
    o.status = r.status == 0 ? SPOCK_OK : (r.status > 0 ? SPOCK_MAXITER : SPOCK_ETIMEOUT);
    o.iters = r.iters;
    o.n_T = r.n_T;
    o.res_inf = r.res_inf;
    o.risk = r.risk;
    memset(o.u0, 0, sizeof(o.u0));
    memcpy(o.u0, r.u0, sizeof(double) * s->plants[p]->nu);
    o.device_ms = 1e-6 * (double)(r.t_done - r.t_claim);
    o.latency_ms = 1e-3 * (double)std::chrono::duration_cast<std::chrono::microseconds>(
                               Clock::now() - s->slot_submit[slot]).count();
    s->slot_busy[slot] = 0;
    s->plant_busy[p] = 0;
    s->outstanding -= 1;
  }
  // requests waiting for a plant that is free now
  for (int p = 0; p < s->count; ++p) {
    if (s->plant_busy[p] || s->queue[p].empty()) continue;
    if (!publish(s, p, s->queue[p].front())) break;
    s->queue[p].pop_front();
  }
  if (n_out) *n_out = n;
  release_evicted(s, false);
  // work left: make sure the persistent launch is there to take it
  return s->outstanding > 0 ? ensure_running(s) : SPOCK_OK;
}

int spock_server_evict(spock_server* s, int plant) {
  if (!s || plant < 0 || plant >= s->count) return SPOCK_EINVAL;
  if (!s->is_admitted[plant]) return SPOCK_OK;
  if (s->plant_busy[plant] || !s->queue[plant].empty()) return SPOCK_EINVAL;   // requests outstanding
  s->is_admitted[plant] = 0;
  if (s->budget > 0) s->room += s->charged[plant];
  s->charged[plant] = 0;
  s->admitted -= 1;
  s->release_pending[plant] = 1;
  release_evicted(s, false);
  return SPOCK_OK;
}

int spock_server_admitted(const spock_server* s, int plant) {
  if (!s || plant < 0 || plant >= s->count) return SPOCK_EINVAL;
  return s->is_admitted[plant] ? 1 : 0;
}

long long spock_server_outstanding(const spock_server* s) { return s ? s->outstanding : -1; }

void spock_server_destroy(spock_server* s) {
  if (!s) return;
  if (s->h_ctl) s->h_ctl->stop = 1;
  if (s->stream) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  release_evicted(s, true);
  if (s->h_ring) cudaFreeHost(s->h_ring);
  if (s->h_res) cudaFreeHost(s->h_res);
  if (s->h_ctl) cudaFreeHost((void*)s->h_ctl);
  s->mem.free_all();
  delete s;
}

}  // extern "C"
