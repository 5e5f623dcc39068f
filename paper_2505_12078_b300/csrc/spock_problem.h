// spock_problem.h -- host-side state of a problem (internal to libspock).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "spock_dev.cuh"
#include "spock_internal.h"

namespace spock {

constexpr int kThreads = 256;

inline int pad4(int x) { return (x + 3) & ~3; }

struct DevMem {
  std::vector<void*> ptrs;
  bool failed = false;
  long long bytes = 0;   // bytes requested by the allocations held
  template <class T>
  T* alloc(long long count) {
    if (count <= 0) count = 1;
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)count * sizeof(T)) != cudaSuccess) {
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    bytes += count * (long long)sizeof(T);
    return static_cast<T*>(p);
  }
  void free_all() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
};

// bytes of one mailbox of the whole-CTA sweeps: n nodes x w values, one
// 64-bit word per 32-bit piece of a value (es: bytes per value)
inline size_t mailbox_bytes(int n, int w, size_t es) { return (size_t)n * (size_t)w * (es / 4) * 8; }

template <class T>
struct Iter {   // per-precision iteration data
  T *MB = nullptr, *MF = nullptr, *MP = nullptr, *KT = nullptr, *cvec = nullptr, *kc = nullptr;
  T *qh = nullptr, *rh = nullptr, *qNh = nullptr, *gx = nullptr, *gu = nullptr, *gN = nullptr;
  T *box_lo = nullptr, *box_hi = nullptr, *boxN_lo = nullptr, *boxN_hi = nullptr, *ball = nullptr;
  T *prob = nullptr, *avar = nullptr, *x0s = nullptr;
  T *qbuf = nullptr, *dbuf = nullptr, *hbuf = nullptr, *ebuf = nullptr;
  T *smw = nullptr, *slo = nullptr;                   // [nx + nu] soft costs: 1/s and -s z_max
  T* tvr = nullptr;                                   // [n_nl] total-variation radii (tv problems)
  T* l1w = nullptr;                                   // [nx + nu] weights 1/s of the l1 row theta - sum
  unsigned long long *mbb = nullptr, *mbf = nullptr;   // sweep mailboxes (whole-CTA sweeps only)
  size_t mb_bytes = 0;                                 // bytes of each
  // full weights, cone translations, general rows (see Prob)
  T *FQ = nullptr, *FQT = nullptr, *FR = nullptr, *FRT = nullptr, *FN = nullptr, *FNT = nullptr;
  T *acost = nullptr, *acostN = nullptr;
  T *Gg = nullptr, *GgT = nullptr, *GgN = nullptr, *GgNT = nullptr;
  T *gen_lo = nullptr, *gen_hi = nullptr, *genN_lo = nullptr, *genN_hi = nullptr;
  // whole-CTA sweeps: output-column-major factors and their layout
  T *MBt = nullptr, *MFt = nullptr, *KTt = nullptr;
  int cta = 0, ldTB = 0, ldTF = 0, ldTK = 0, khB = 0, khF = 0, nbuf = 0, item_bytes = 0, qslots = 0,
      ldc = 0;
  SolveBufs<T> sb{};
  bool have_bufs = false;
  void* sb_block = nullptr;   // the one device allocation that holds every buffer of sb
  Prob<T> P{};
};


}  // namespace spock

struct spock_problem {
  int n = 0, n_nl = 0, n_l = 0, N = 0, nx = 0, nu = 0, n_c = 0, n_cN = 0;
  int nbx = 0, nbu = 0, nbox = 0, has_ball = 0;
  int full = 0;        // Q, R, QN given as full matrices
  int has_lin = 0;     // some linear cost term present
  int n_g = 0, n_gN = 0;   // general constraint rows (non-leaf, leaf)
  double l1 = 0.0;         // lambda_0 of the l1 edge-cost term (Prop. 2), 0 = none
  int tv = 0;              // 1: total-variation risks (radius per non-leaf node in tvr), 0: AV@R
  int soft = 0;            // soft-constraint costs (the penalty after Prop. 2)
  std::vector<double> soft_max;
  long long o_sg = 0, o_sth = 0, e_sf = 0;   // their blocks: sigma, theta in z; their rows in eta
  std::vector<double> tvr;
  long long o_th = 0, o_lam = 0, e_l1 = 0;   // its blocks: theta, lambda in z; its rows in eta
  long long n_y = 0, nz = 0, neta = 0, nv = 0;
  long long o_x, o_u, o_y, o_tau, o_s, e_y, e_s, e_c, e_q, e_cN, e_qN;
  int ldB, ldF, ldP, ldK;
  std::vector<int> anc, ch_off, yoff, stage_off, ynode, lvl_off, seg_top, seg_bot, seg_len, seg_off,
      seg_nodes;
  std::vector<double> Sx, Su, SxN;
  double a_con = 1, a_conN = 1, alpha = 0, normL = 0;
  int max_items = 1;
  int maxch = 1;       // most children of a node
  int tw = 8;
  int use_pipe = 1;    // stream the sweep matrices through shared memory
  spock::DevMem mem;
  // device tree / schedule
  int *d_anc, *d_ch_off, *d_yoff, *d_ynode, *d_lvl_off, *d_seg_top, *d_seg_bot, *d_seg_len,
      *d_seg_off, *d_seg_nodes;
  int4* d_seg_info;
  int *d_top_seg, *d_bot_seg;   // segment of a top / bottom node (or -1)
  // FP64 offline data kept for inspection
  double *d_P, *d_K, *d_Rt, *d_Abar, *d_Sx, *d_SxN, *d_Su;
  double* d_x0raw;   // unscaled x0 of the operator-level calls
  spock::Iter<double> f64;
  spock::Iter<float> f32;
  double* d_out_risk;
  double* d_diag_part = nullptr;   // partials and result of the FP64 exit check (first use)
  long long setup_peak = 0;        // device bytes held at the end of the offline part (its peak)
  // centred FP32 iteration (first use): the centre's eta data A, B (FP64,
  // n_eta each), cz (FP32, n_z) and zeros standing in for the constant terms
  void* ctr_block = nullptr;
  long long ctr_bytes = 0;
  double *d_ctrA = nullptr, *d_ctrB = nullptr;
  float *d_cz = nullptr, *d_zero32 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace spock {
// solve buffers of one precision, allocated on first use
template <class T>
int ensure_bufs(spock_problem* p, Iter<T>& it);
// bytes of one precision's solve buffers (one allocation: seven n_v vectors,
// the Anderson memory S and Y, reduction partials, barrier and segment flags,
// the control block)
long long solve_buffer_bytes(const spock_problem* p, int precision);
// free one precision's solve buffers (the next solve allocates them again and
// starts cold); the caller makes sure no kernel uses them
template <class T>
void release_bufs(Iter<T>& it);
// FP64 exit check of an iterate v (device, `precision` 32 or 64): T(v) in FP64,
// then ||v - T(v)||_inf, xi1, xi2, infeasibility, gap, <eta+, L z+> and
// sigma_S3(eta+) into out7 (host). Uses the problem's FP64 solve buffers VT,
// TVT, VP, RP and S as scratch. Blocking.
int check_fp64(spock_problem* p, int precision, const void* v, cudaStream_t st, double* out7);
}  // namespace spock
