// spock_cta.cuh -- the backward and forward sweeps of Alg. 2 over one segment
// (a chain of single-child nodes whose bottom node has any number of
// children), run by a whole CTA of 256 threads when nx + nu <= 128.
//
// Thread t owns output column t/2 and half t%2 of that column's rows. The
// factors are stored output-column-major (MBt, MFt, KTt), so each thread
// reads its rows with 16-byte shared loads, and the two halves are combined
// by one shuffle. An "item" is one factor matrix (backward: MB of a child;
// forward: [KT of the node | MF of the child], either part alone where the
// other has no output; see "item issue" below for the item lists); items
// stream through a ring of nbuf shared buffers by cp.async.bulk, up to
// nbuf - 1 items ahead of the one in use. Each item ends with one CTA barrier,
// which both publishes the carry vector written in its epilogue and frees the
// buffer of the previous item for the next copy.
//
// Per CTA, the segments it sweeps (the same in every evaluation of T) are
// listed once per launch in shared memory with their node lists (Sched).
#pragma once

#include "spock_dev.cuh"

// Optional cycle trace of CTA 0, thread 0 (compiled in only with
// SPOCK_TRACE_ON, which also provides spock_trace(int point)).
#ifdef SPOCK_TRACE_ON
#define SPOCK_TRACE(k) spock_trace(k)
#else
#define SPOCK_TRACE(k) ((void)0)
#endif
// cycle probe of the sweeps into the launch's probe slots 8..11 (off unless
// SPOCK_PROBE is defined: it costs CTA 0 a few instructions per item)
#ifdef SPOCK_PROBE
#define SPOCK_PROBE_ON true
#else
#define SPOCK_PROBE_ON false
#endif

namespace spock {

// 16-byte shared loads and stores at 32-bit shared addresses
template <class T>
struct SV;
template <>
struct SV<float> {
  static constexpr int W = 4;
};
template <>
struct SV<double> {
  static constexpr int W = 2;
};
__device__ __forceinline__ void ld16(unsigned a, float (&v)[4]) {
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "r"(a));
}
__device__ __forceinline__ void ld16(unsigned a, double (&v)[2]) {
  asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
}
template <class T>
__device__ __forceinline__ T ld_s(unsigned a);
template <>
__device__ __forceinline__ float ld_s<float>(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
template <>
__device__ __forceinline__ double ld_s<double>(unsigned a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
template <class T>
__device__ __forceinline__ void st_s(unsigned a, T v);
template <>
__device__ __forceinline__ void st_s<float>(unsigned a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
template <>
__device__ __forceinline__ void st_s<double>(unsigned a, double v) {
  asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// sum_k m[k] x[k] over ng 16-byte groups of rows at shared addresses m and x;
// rows past the last real row of a group are zero in m (column padding) and
// finite in x. Groups of eight are unrolled with a predicate, which lets the
// loads of a group be issued ahead of the previous group's FMAs.
template <class T>
__device__ __forceinline__ T tdot(unsigned m, unsigned x, int ng) {
  constexpr int W = SV<T>::W;
  T a[W];
#pragma unroll
  for (int w = 0; w < W; ++w) a[w] = T(0);
  for (int g0 = 0; g0 < ng; g0 += 8) {
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      if (g0 + g < ng) {
        T mv[W], xv[W];
        ld16(m + 16u * (unsigned)(g0 + g), mv);
        ld16(x + 16u * (unsigned)(g0 + g), xv);
#pragma unroll
        for (int w = 0; w < W; ++w) a[w] = fma(mv[w], xv[w], a[w]);
      }
    }
  }
  if constexpr (W == 4)
    return (a[0] + a[1]) + (a[2] + a[3]);
  else
    return a[0] + a[1];
}

// ---------------------------------------------------------------------------
// The item ring: nbuf buffers, one mbarrier each (8 bytes apart). The state
// persists across segments and evaluations; the sweeps copy it to registers.
// ---------------------------------------------------------------------------
struct Ring {
  unsigned bar0;     // shared address of mbarrier 0
  unsigned buf0;     // shared address of buffer 0
  unsigned bstride;  // bytes per buffer
  int nbuf;
  unsigned par;      // bit b: parity of the next phase of buffer b's mbarrier
  int head;          // buffer of the next item to be waited for
  int ahead;         // items of the next segment already issued
  int* diag;
  __device__ __forceinline__ unsigned bar(int b) const { return bar0 + 8u * (unsigned)b; }
  __device__ __forceinline__ unsigned buf(int b) const { return buf0 + bstride * (unsigned)b; }
  __device__ __forceinline__ int step(int b, int k) const {   // (b + k) mod nbuf, 0 <= k < nbuf
    b += k;
    return b >= nbuf ? b - nbuf : b;
  }
};
__device__ __forceinline__ void ring_arm(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void ring_copy(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// thread 0 waits (bounded) for the item in buffer b; every thread flips the
// buffer's parity. The caller's CTA barrier hands the verdict (*s_ok) on.
__device__ __forceinline__ void ring_wait0(Ring& R, int b, int* err, int site, int* s_ok) {
  if (threadIdx.x == 0) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(__cvta_shared_to_generic(R.bar(b)));
    if (!mbar_wait(bar, (R.par >> b) & 1u, err, R.diag, site)) *s_ok = 0;
  }
  R.par ^= 1u << b;
}

// ---------------------------------------------------------------------------
// Per-CTA list of segments, level by level (same order in every evaluation)
// ---------------------------------------------------------------------------
constexpr int SCHED_CAP = 1536;   // ints of records
constexpr int SCHED_LEV = 64;     // levels
constexpr int SEG_HDR = 5;        // s, len, first child, one past last child, list offset
struct Sched {
  int ok;                    // every record of this CTA fits
  int lvl[SCHED_LEV + 1];    // offset of the first record of level l
  int rec[SCHED_CAP];        // per segment: header, then its nodes top to bottom
};

struct SegRef {
  int s, len, c0, c1;
  const int* nodes;          // shared (from Sched) or global (seg_nodes)
};

// build the schedule of this CTA (team index tg of nt); every thread calls it
template <class T>
__device__ void sched_build(const Prob<T>& P, Sched& S, int tg, int nt) {
  const int L = P.n_levels;
  if (threadIdx.x == 0) {
    int off = 0;
    bool ok = L <= SCHED_LEV;
    for (int l = 0; l < L && ok; ++l) {
      S.lvl[l] = off;
      for (int s = P.lvl_off[l] + tg; s < P.lvl_off[l + 1]; s += nt) {
        const int4 inf = P.seg_info[s];
        if (off + SEG_HDR + inf.y > SCHED_CAP) { ok = false; break; }
        S.rec[off] = s; S.rec[off + 1] = inf.y; S.rec[off + 2] = inf.z; S.rec[off + 3] = inf.w;
        S.rec[off + 4] = inf.x;
        off += SEG_HDR + inf.y;
      }
    }
    if (ok) S.lvl[L] = off;
    S.ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (S.ok) {
    for (int r = 0; r < S.lvl[L];) {
      const int len = S.rec[r + 1], go = S.rec[r + 4];
      for (int k = threadIdx.x; k < len; k += blockDim.x) S.rec[r + SEG_HDR + k] = P.seg_nodes[go + k];
      r += SEG_HDR + len;
    }
  }
  __syncthreads();
}

// number of this CTA's segments in level l
template <class T>
__device__ __forceinline__ int seg_count(const Prob<T>& P, int l, int tg, int nt) {
  const int m = P.lvl_off[l + 1] - P.lvl_off[l] - tg;
  return m > 0 ? (m + nt - 1) / nt : 0;
}
// the k-th segment of this CTA in level l
template <class T>
__device__ __forceinline__ SegRef seg_get(const Prob<T>& P, const Sched& S, int l, int k, int tg, int nt) {
  SegRef r;
  if (S.ok) {
    int o = S.lvl[l];
    for (int q = 0; q < k; ++q) o += SEG_HDR + S.rec[o + 1];
    r.s = S.rec[o]; r.len = S.rec[o + 1]; r.c0 = S.rec[o + 2]; r.c1 = S.rec[o + 3];
    r.nodes = S.rec + o + SEG_HDR;
  } else {
    r.s = P.lvl_off[l] + tg + k * nt;
    const int4 inf = P.seg_info[r.s];
    r.len = inf.y; r.c0 = inf.z; r.c1 = inf.w;
    r.nodes = P.seg_nodes + inf.x;
  }
  return r;
}

// the shared areas of the whole-CTA sweeps (32-bit addresses)
struct CtaMem {
  unsigned carry0, carry1;   // carry vectors (ldc elements each)
  unsigned qin;              // child inputs of a backward bottom (qslots x ldc)
};

// everything the whole-CTA sweeps keep between segments and evaluations
struct CtaState {
  Ring ring;
  CtaMem mem;
  const Sched* sched;
  int* s_ok;
  unsigned* seg_flags;   // per-segment flags (zeroed at launch; the sweeps hand over
                         // through the tagged mailboxes instead)
  unsigned epoch;        // evaluations of T so far in this launch; the sweep tags
                         // are 2 epoch (backward) and 2 epoch + 1 (forward)
};

// Dataflow between the sweeps' levels: a segment's backward sweep waits for
// the shares of the segments headed by its bottom's children, its forward
// sweep for the [x; d] of the segment that ends in its top's parent, both
// through tagged mailboxes (below). The waits point to deeper (backward) or
// higher (forward) levels, which every CTA sweeps first, so they cannot form
// a cycle. Every wait is bounded.
// after a failed wait: let the copies already issued into the ring land
// (bounded) before the CTA leaves
__device__ __forceinline__ void ring_settle(Ring& R, int issued) {
  if (threadIdx.x == 0) {
    for (int j = 0; j < issued; ++j) {
      const int b = R.step(R.head, j);
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(reinterpret_cast<uint64_t*>(__cvta_shared_to_generic(R.bar(b))), (R.par >> b) & 1u) &&
             global_ns() - t0 < 200000000ull) {
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Mailboxes between the CTAs of the sweeps. Every 32-bit piece of a value goes
// into one 64-bit word beside a 32-bit tag (the sweep epoch of the current
// evaluation: 2e backward, 2e + 1 forward; the mailboxes are zeroed before a
// launch and e >= 1, so no stale word carries a current tag). A 64-bit word
// is written and read in one access, so a reader that sees the tag also sees
// the value: the hand-over between segments needs neither a fence nor a
// separate flag, and costs one round trip to L2 once the value has landed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mb_st64(unsigned long long* p, unsigned tag, unsigned bits) {
  const unsigned long long v = ((unsigned long long)tag << 32) | (unsigned long long)bits;
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long mb_ld64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
template <class T>
struct MB;
template <>
struct MB<float> {
  static constexpr int WPV = 1;   // words per value
  static __device__ __forceinline__ void put(unsigned long long* p, float v, unsigned tag) {
    mb_st64(p, tag, __float_as_uint(v));
  }
  static __device__ __forceinline__ bool get(const unsigned long long* p, unsigned tag, float& v) {
    const unsigned long long w = mb_ld64(p);
    if ((unsigned)(w >> 32) != tag) return false;
    v = __uint_as_float((unsigned)w);
    return true;
  }
};
template <>
struct MB<double> {
  static constexpr int WPV = 2;
  static __device__ __forceinline__ void put(unsigned long long* p, double v, unsigned tag) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    mb_st64(p, tag, (unsigned)b);
    mb_st64(p + 1, tag, (unsigned)(b >> 32));
  }
  static __device__ __forceinline__ bool get(const unsigned long long* p, unsigned tag, double& v) {
    const unsigned long long lo = mb_ld64(p), hi = mb_ld64(p + 1);
    if ((unsigned)(lo >> 32) != tag || (unsigned)(hi >> 32) != tag) return false;
    v = __longlong_as_double((long long)((hi << 32) | (lo & 0xffffffffull)));
    return true;
  }
};
// wait (bounded, as the barriers) until the word(s) at p carry tag; false on
// a timeout or when the launch is already failing
template <class T>
__device__ __forceinline__ bool mb_wait(const unsigned long long* p, unsigned tag, T& v, int* err) {
  uint64_t t0 = 0;
  unsigned spins = 0;
  while (!MB<T>::get(p, tag, v)) {
    if (++spins > 32u) __nanosleep(32);
    if ((spins & 31u) == 0u) {
      if (ld_relaxed_i(err)) return false;
      const uint64_t t = global_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > BARRIER_LIMIT_NS) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
  return true;
}

// dynamic shared memory of the whole-CTA sweeps: the ring, two carry vectors
// and the child inputs
template <class T>
__host__ __device__ inline size_t cta_smem_bytes(const Prob<T>& P) {
  if (!P.cta) return 0;
  return (size_t)P.nbuf * P.item_bytes + (size_t)(2 + P.qslots) * P.ldc * sizeof(T);
}

// ---------------------------------------------------------------------------
// item issue (by one thread)
//
// The items of a segment. A node's children that head segments of their own
// (its non-leaf children) are not items of the node's segment: in the
// backward sweep every segment ends with an uplink item that forms its top's
// share of the parent's step, MB_top' v_top, and the parent adds these shares;
// in the forward sweep every segment starts with a downlink item that forms
// its top's state from the parent's [x; d]. The children of a branching node
// therefore run their items on their own CTAs at the same time, and the
// parent's segment has no per-child item left on the critical path.
//   backward: the bottom's leaf children (inputs from phase P), one item per
//             step up the chain, then the uplink (not for the root);
//   forward:  the downlink (not for the root), one item per step down the
//             chain ([KT_i | MF_child]), then the bottom's leaf children
//             ([KT | MF] for the first, MF for the rest), or KT alone when the
//             bottom has no leaf child.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int seg_leaf0(const Prob<T>& P, const SegRef& g) {   // first leaf child of the bottom
  return max(g.c0, P.n_nl);
}
template <class T>
__device__ __forceinline__ int seg_nleaf(const Prob<T>& P, const SegRef& g) {   // leaf children of the bottom
  return max(0, g.c1 - max(g.c0, P.n_nl));
}
template <class T>
__device__ __forceinline__ int b_items(const Prob<T>& P, const SegRef& g) {
  return seg_nleaf(P, g) + g.len - 1 + (g.nodes[0] != 0 ? 1 : 0);
}
template <class T>
__device__ __forceinline__ int f_items(const Prob<T>& P, const SegRef& g) {
  return (g.nodes[0] != 0 ? 1 : 0) + g.len - 1 + max(1, seg_nleaf(P, g));
}
// the child whose MB the backward item j uses
template <class T>
__device__ __forceinline__ int b_child(const Prob<T>& P, const SegRef& g, int j) {
  const int nbl = seg_nleaf(P, g);
  if (j < nbl) return seg_leaf0(P, g) + j;
  j -= nbl;
  return (j < g.len - 1) ? g.nodes[g.len - 1 - j] : g.nodes[0];
}
// what the issuing thread needs, read from the problem once per segment
template <class T>
struct BIssue {
  const T* base;     // MBt
  size_t stride;     // elements per child
  unsigned bytes;
  __device__ __forceinline__ explicit BIssue(const Prob<T>& P)
      : base(P.MBt), stride((size_t)(P.nx + P.nu) * P.ldTB), bytes((unsigned)((P.nx + P.nu) * P.ldTB * (int)sizeof(T))) {}
};
template <class T>
__device__ __forceinline__ void b_issue(const Prob<T>& P, const BIssue<T>& I, const Ring& R, const SegRef& g, int j,
                                        int b) {
  const int c = b_child(P, g, j);
  const bool ok = SPOCK_CHK(c >= 1 && c < P.n, 1);   // (a failed check arms no bytes: the slot completes empty)
  ring_arm(R.bar(b), ok ? I.bytes : 0u);
  if (ok) ring_copy(R.buf(b), I.base + (size_t)(c - 1) * I.stride, I.bytes, R.bar(b));
}
// forward item j: the node whose [x; d] is the input, the child whose x is an
// output (-1: none), and whether the node's u (KT) is an output
template <class T>
__device__ __forceinline__ void f_item(const Prob<T>& P, const SegRef& g, int j, int& node, int& child, bool& kt) {
  const int top = g.nodes[0];
  if (top != 0) {
    if (j == 0) { node = -1; child = top; kt = false; return; }   // downlink (node: the parent)
    --j;
  }
  if (j < g.len - 1) {
    node = g.nodes[j]; child = g.nodes[j + 1]; kt = true;
    return;
  }
  j -= g.len - 1;
  node = g.nodes[g.len - 1];
  const int nbl = seg_nleaf(P, g);
  child = (nbl > 0) ? seg_leaf0(P, g) + j : -1;
  kt = (j == 0);
}
template <class T>
struct FIssue {
  const T* kt;       // KTt
  const T* mf;       // MFt
  size_t ks, fs;     // elements per node / per child
  unsigned kb, fb;   // bytes of the two parts
  __device__ __forceinline__ explicit FIssue(const Prob<T>& P)
      : kt(P.KTt), mf(P.MFt), ks((size_t)P.nu * P.ldTK), fs((size_t)P.nx * P.ldTF),
        kb((unsigned)(P.nu * P.ldTK * (int)sizeof(T))), fb((unsigned)(P.nx * P.ldTF * (int)sizeof(T))) {}
};
// the buffer holds [KT part | MF part], the MF part at byte offset kb
template <class T>
__device__ __forceinline__ void f_issue(const Prob<T>& P, const FIssue<T>& I, const Ring& R, const SegRef& g, int j,
                                        int b) {
  int node, child;
  bool kt;
  f_item(P, g, j, node, child, kt);
  const bool okk = !kt || SPOCK_CHK(node >= 0 && node < P.n_nl, 2);
  const bool okf = child < 0 || SPOCK_CHK(child >= 1 && child < P.n, 2);
  ring_arm(R.bar(b), (kt && okk ? I.kb : 0u) + (child >= 0 && okf ? I.fb : 0u));
  if (kt && okk) ring_copy(R.buf(b), I.kt + (size_t)node * I.ks, I.kb, R.bar(b));
  if (child >= 0 && okf) ring_copy(R.buf(b) + I.kb, I.mf + (size_t)(child - 1) * I.fs, I.fb, R.bar(b));
}
// first items of the next segment (backward or forward), issued ahead of its call
template <class T>
__device__ __forceinline__ void ring_prefetch(const Prob<T>& P, Ring& R, const SegRef& g, bool fwd) {
  const int nitems = fwd ? f_items(P, g) : b_items(P, g);
  const int k = min(R.nbuf - 1, nitems);
  if (threadIdx.x == blockDim.x - 1) {
    if (fwd) {
      const FIssue<T> I(P);
      for (int j = 0; j < k; ++j) f_issue(P, I, R, g, j, R.step(R.head, j));
    } else {
      const BIssue<T> I(P);
      for (int j = 0; j < k; ++j) b_issue(P, I, R, g, j, R.step(R.head, j));
    }
  }
  R.ahead = k;
}

// ---------------------------------------------------------------------------
// backward sweep of one segment:
//   v_c = q_c + P_c c_c (q_c holds it, see phase P);  q^i = sum_c Abar_c' v_c + h^i;
//   d^i = e^i - sum_c (B_c Rt_i^{-1})' v_c
// items: the bottom's leaf children, one per step up the chain, then the
// uplink (the top's share MB_top' v_top of its parent's step, into the
// mailbox mbb); the shares of the bottom's non-leaf children come from their
// segments' uplinks
// ---------------------------------------------------------------------------
template <class T>
__device__ bool bwd_cta(const Prob<T>& P, const CtaMem& cm, Ring& ring, int* err, const SegRef& g,
                        int* s_ok, unsigned long long* prof, unsigned* flags, unsigned eB) {
  constexpr int W = SV<T>::W;
  constexpr unsigned ES = sizeof(T);
  const int nx = P.nx, nu = P.nu, w = nx + nu;
  const int t = threadIdx.x, col = t >> 1, half = t & 1;
  const bool has_col = col < w;
  const bool owner = has_col && !half;   // writes the column's result
  const bool issuer = (t == (int)blockDim.x - 1);
  const int r0 = half ? P.khB : 0;
  const int r1 = half ? nx : min(P.khB, nx);
  const int ng = (has_col && r1 > r0) ? (r1 - r0 + W - 1) / W : 0;
  const unsigned mcol = (unsigned)(col * P.ldTB + r0) * ES;
  const unsigned xoff = (unsigned)r0 * ES;
  const unsigned ldcb = (unsigned)P.ldc * ES;
  T* __restrict__ qbuf = P.qbuf;
  T* __restrict__ dbuf = P.dbuf;
  const T* __restrict__ hbuf = P.hbuf;
  const T* __restrict__ ebuf = P.ebuf;
  Ring R = ring;
  const BIssue<T> I(P);
  const int len = g.len, QS = P.qslots, top = g.nodes[0];
  const int nbl = seg_nleaf(P, g), leaf0 = seg_leaf0(P, g);
  const int nbn = max(0, min(g.c1, P.n_nl) - g.c0);   // non-leaf children: shares from their uplinks
  const int nchain = len - 1;
  const int nitems = nbl + nchain + (top != 0 ? 1 : 0);
  const bool probe = SPOCK_PROBE_ON && prof && blockIdx.x == 0 && t == 0;
  long long tc = probe ? clock64() : 0, c_mv = 0, c_hand = 0;
  // the items not issued ahead, up to nbuf - 1 in flight
  if (issuer)
    for (int j = R.ahead; j < min(R.nbuf - 1, nitems); ++j) b_issue(P, I, R, g, j, R.step(R.head, j));
  R.ahead = 0;
  if (t == 0) *s_ok = 1;
  __syncthreads();
  // h/e of the output nodes (bottom first, then up the chain), two ahead
  auto pre_of = [&](int node) -> T {
    if (!owner) return T(0);
    return (col < nx) ? ldc(hbuf + (long long)node * nx + col) : ldc(ebuf + (long long)node * nu + (col - nx));
  };
  T preA = pre_of(g.nodes[len - 1]);
  T preB = (len >= 2) ? pre_of(g.nodes[len - 2]) : T(0);
  // the shares of the bottom's non-leaf children, from their segments'
  // uplinks (mailbox mbb), summed in child order
  T share = T(0);
  if (owner) {
    for (int c = g.c0; c < g.c0 + nbn; ++c) {
      T sv;
      if (!SPOCK_CHK(c >= 1 && c < P.n_nl, 3) ||
          !mb_wait<T>(P.mbb + ((long long)c * w + col) * MB<T>::WPV, eB, sv, err)) {
        *s_ok = 0;
        break;
      }
      share += sv;
    }
  }
  // inputs of the bottom's first leaf children
  auto load_children = [&](int j0) {
    const int m = min(QS, nbl - j0);
    for (int e = t; e < m * nx; e += blockDim.x) {
      const int j = e / nx, k = e - j * nx;
      if (SPOCK_CHK(leaf0 + j0 + j >= P.n_nl && leaf0 + j0 + j < P.n, 5))
        st_s<T>(cm.qin + (unsigned)j * ldcb + (unsigned)k * ES, ldc(qbuf + (long long)(leaf0 + j0 + j) * nx + k));
    }
  };
  if (nbl > 0) load_children(0);
  unsigned cin = cm.carry0, cout = cm.carry1;
  int nout = 0;   // output nodes done (bottom = 0, then up the chain)
  auto epilogue = [&](T s) {
    const int i = g.nodes[len - 1 - nout];
    if (owner && SPOCK_CHK(i >= 0 && i < P.n_nl, 4)) {
      if (col < nx) {
        const T qq = s + preA;
        st_s<T>(cout + (unsigned)col * ES, qq);
        stc(qbuf + (long long)i * nx + col, qq);
      } else {
        stc(dbuf + (long long)i * nu + (col - nx), preA - s);
      }
    }
    ++nout;
    preA = preB;
    preB = (len - 2 - nout >= 0) ? pre_of(g.nodes[len - 2 - nout]) : T(0);
    const unsigned tt = cin; cin = cout; cout = tt;
  };
  if (nbl == 0) epilogue(share);   // the bottom's step is its children's shares alone
  int b = R.head;
  if (nitems > 0) ring_wait0(R, b, err, 3, s_ok);
  __syncthreads();
  bool ok = *s_ok != 0;
  if (!ok) {   // let the other copies in flight land before the CTA leaves
    if (nitems > 1) {
      R.head = R.step(b, 1);
      ring_settle(R, min(R.nbuf - 1, nitems) - 1);
    }
    ring = R;
    return false;
  }
  T acc = T(0);
  for (int j = 0; j < nitems && ok; ++j) {
    // next copy into the buffer of item j - 1 (freed by the barrier that ended it)
    if (issuer && j + R.nbuf - 1 < nitems) b_issue(P, I, R, g, j + R.nbuf - 1, R.step(b, R.nbuf - 1));
    if (j < nbl && j > 0 && j % QS == 0) {   // next chunk of the bottom's leaf children
      load_children(j);
      __syncthreads();
    }
    const unsigned xin = (j < nbl) ? cm.qin + (unsigned)(j % QS) * ldcb : cin;
    if (probe) { const long long c = clock64(); c_hand += c - tc; tc = c; }
    T v = (ng > 0) ? tdot<T>(R.buf(b) + mcol, xin + xoff, ng) : T(0);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    acc += v;
    if (j < nbl) {
      if (j == nbl - 1) {
        epilogue(acc + share);
        acc = T(0);
      }
    } else if (j < nbl + nchain) {
      epilogue(acc);
      acc = T(0);
    } else {   // uplink: the top's share of its parent's step, to the parent's segment
      if (owner && SPOCK_CHK(top >= 1 && top < P.n_nl, 3))
        MB<T>::put(P.mbb + ((long long)top * w + col) * MB<T>::WPV, acc, eB);
      acc = T(0);
    }
    if (probe) { const long long c = clock64(); c_mv += c - tc; tc = c; }
    b = R.step(b, 1);
    if (j + 1 < nitems) ring_wait0(R, b, err, 3, s_ok);
    __syncthreads();
    ok = *s_ok != 0;
  }
  if (probe) {
    const long long c = clock64();
    c_hand += c - tc;
    prof[8] += (unsigned long long)c_hand;
    prof[9] += (unsigned long long)c_mv;
  }
  R.head = b;
  ring = R;
  return ok;
}

// ---------------------------------------------------------------------------
// forward rollout of one segment:  u^i = K_i x^i + d^i;  x^c = Abar_c x^i + B_c d^i + c_c
// items: the downlink (x of the top from its parent's [x; d]), one per step
// down the chain (KT_i with the child's MF), then the bottom's leaf children
// (KT of the bottom with the first), or KT alone; the input of an item is
// [x; d] of its node in the carry vector. [x; d] of the bottom goes to the
// mailbox as soon as x of the bottom is known, so that the segments of its
// non-leaf children start while this one finishes u of the bottom and the
// leaves.
// ---------------------------------------------------------------------------
template <class T>
__device__ bool fwd_cta(const Prob<T>& P, const CtaMem& cm, Ring& ring, int* err, const SegRef& g,
                        T* __restrict__ vout, int* s_ok, unsigned long long* prof, unsigned* flags,
                        unsigned eF) {
  constexpr int W = SV<T>::W;
  constexpr unsigned ES = sizeof(T);
  const int nx = P.nx, nu = P.nu, w = nx + nu;
  const int t = threadIdx.x;
  // x columns run over the nx + nu rows of MFt, u columns over the nx rows of
  // KTt. In FP32, when 4 nx + 2 nu threads fit, an x column gets four threads
  // (a quarter of its rows each) and a u column two, which evens out the two
  // critical paths. Otherwise (and in FP64, whose items are bound by the FP64
  // pipe and whose column layout is tuned for two threads) two threads per
  // column of either kind.
  const int XP = (sizeof(T) == 4 && 4 * nx + 2 * nu <= (int)blockDim.x) ? 4 : 2;
  const int nxt = XP * nx;
  const bool xcol = t < nxt, ucol = !xcol && t < nxt + 2 * nu;
  const int col = xcol ? t / XP : (ucol ? nx + ((t - nxt) >> 1) : w);
  const int part = xcol ? t % XP : ((t - nxt) & 1);
  const bool lead = part == 0;   // the thread that writes the column's result
  const bool issuer = (t == (int)blockDim.x - 1);
  int r0 = 0, r1 = 0;
  if (xcol && XP == 4) {
    const int kq = ((w + 3) / 4 + W - 1) / W * W;   // rows per quarter, whole 16-byte groups
    r0 = part * kq;
    r1 = min(r0 + kq, w);
  } else if (xcol) {
    r0 = part ? P.khF : 0;
    r1 = part ? w : min(P.khF, w);
  } else if (ucol) {
    r0 = part ? P.khB : 0;
    r1 = part ? nx : min(P.khB, nx);
  }
  const int ng = ((xcol || ucol) && r1 > r0) ? (r1 - r0 + W - 1) / W : 0;
  const unsigned kbytes = (unsigned)(nu * P.ldTK) * ES;
  const unsigned mcol = xcol ? kbytes + (unsigned)(col * P.ldTF + r0) * ES
                             : (unsigned)((col - nx) * P.ldTK + r0) * ES;
  const unsigned xoff = (unsigned)r0 * ES;
  const T* __restrict__ dbuf = P.dbuf;
  const T* __restrict__ cvec = P.cvec;
  const long long o_x = P.o_x, o_u = P.o_u;
  Ring R = ring;
  const FIssue<T> I(P);
  const int len = g.len, top = g.nodes[0];
  const int down = (top != 0) ? 1 : 0;
  const int ncont = down + len - 1;   // items whose child is the next item's node
  const int nitems = ncont + max(1, seg_nleaf(P, g));
  // x of the bottom is stored by item jx (-1: before the first item)
  const int jx = ncont - 1;
  const bool probe = SPOCK_PROBE_ON && prof && blockIdx.x == 0 && t == 0;
  long long tc = probe ? clock64() : 0, c_mv = 0, c_hand = 0;
  if (issuer)
    for (int j = R.ahead; j < min(R.nbuf - 1, nitems); ++j) f_issue(P, I, R, g, j, R.step(R.head, j));
  R.ahead = 0;
  const int par = down ? P.anc[top] : 0;
  const int bottom = g.nodes[len - 1];
  if (t == 0) *s_ok = 1;
  __syncthreads();
  // c_c of item j's child (x columns), d of the child of a continuing item, two items ahead
  auto child_of = [&](int j) {
    int nd, ch;
    bool kt;
    f_item(P, g, j, nd, ch, kt);
    return ch;
  };
  auto cp_of = [&](int j) -> T {
    if (j >= nitems || !(xcol && lead)) return T(0);
    const int c = child_of(j);
    return c >= 0 ? ldr(cvec + (long long)(c - 1) * nx + col) : T(0);
  };
  auto dn_of = [&](int j) -> T {   // d of the child of continuing item j, element t
    if (!(j < ncont && t < nu)) return T(0);
    const int ch = child_of(j);
    return SPOCK_CHK(ch >= 0 && ch < P.n_nl, 8) ? ldc(dbuf + (long long)ch * nu + t) : T(0);
  };
  T cpA = cp_of(0), cpB = cp_of(1);
  T dA = dn_of(0), dB = dn_of(1);
  // input of the first item: [x; d] of the parent (downlink, from the parent's
  // segment through the mailbox mbf) or of the root
  unsigned cin = cm.carry0, cout = cm.carry1;
  for (int k = t; k < w; k += blockDim.x) {
    T v = T(0);
    if (down) {
      if (!SPOCK_CHK(par >= 0 && par < P.n_nl, 6) ||
          !mb_wait<T>(P.mbf + ((long long)par * w + k) * MB<T>::WPV, eF, v, err)) *s_ok = 0;
    } else if (k < nx) {
      v = P.x0s[k];
      stc(vout + o_x + k, zc_add(P, o_x + k, v));
    } else {
      v = ldc(dbuf + (k - nx));
    }
    st_s<T>(cin + (unsigned)k * ES, v);
  }
  int b = R.head;
  ring_wait0(R, b, err, 4, s_ok);
  __syncthreads();
  bool ok = *s_ok != 0;
  if (!ok) {   // let the other copies in flight land before the CTA leaves
    if (nitems > 1) {
      R.head = R.step(b, 1);
      ring_settle(R, min(R.nbuf - 1, nitems) - 1);
    }
    ring = R;
    return false;
  }
  // [x; d] of the bottom for the segments of its children
  auto publish = [&]() {
    if (t < w && SPOCK_CHK(bottom >= 0 && bottom < P.n_nl, 6))
      MB<T>::put(P.mbf + ((long long)bottom * w + t) * MB<T>::WPV, ld_s<T>(cin + (unsigned)t * ES), eF);
  };
  if (jx < 0) publish();   // the root alone: x0
  for (int j = 0; j < nitems && ok; ++j) {
    if (issuer && j + R.nbuf - 1 < nitems) f_issue(P, I, R, g, j + R.nbuf - 1, R.step(b, R.nbuf - 1));
    int nd, c;
    bool kt;
    f_item(P, g, j, nd, c, kt);
    const bool cont = j < ncont;
    if (probe) { const long long cc = clock64(); c_hand += cc - tc; tc = cc; }
    T v = T(0);
    if (ng > 0 && ((xcol && c >= 0) || (ucol && kt))) v = tdot<T>(R.buf(b) + mcol, cin + xoff, ng);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    {
      const T v2 = __shfl_xor_sync(0xffffffffu, v, 2);   // groups of four are lane-aligned
      if (XP == 4 && xcol) v += v2;
    }
    if (lead) {
      if (xcol && c >= 0 && SPOCK_CHK(c >= 1 && c < P.n, 7)) {
        const T xc = v + cpA;
        const long long ix = o_x + (long long)c * nx + col;
        stc(vout + ix, zc_add(P, ix, xc));
        if (cont) st_s<T>(cout + (unsigned)col * ES, xc);
      } else if (ucol && kt && SPOCK_CHK(nd >= 0 && nd < P.n_nl, 7)) {
        const long long iu = o_u + (long long)nd * nu + (col - nx);
        stc(vout + iu, zc_add(P, iu, v + ld_s<T>(cin + (unsigned)col * ES)));
      }
    }
    if (cont && t < nu) st_s<T>(cout + (unsigned)(nx + t) * ES, dA);
    cpA = cpB;
    cpB = cp_of(j + 2);
    dA = dB;
    dB = dn_of(j + 2);
    if (cont) { const unsigned tt = cin; cin = cout; cout = tt; }
    if (probe) { const long long cc = clock64(); c_mv += cc - tc; tc = cc; }
    b = R.step(b, 1);
    if (j + 1 < nitems) ring_wait0(R, b, err, 4, s_ok);
    __syncthreads();
    ok = *s_ok != 0;
    if (ok && j == jx) publish();   // [x; d] of the bottom is in the carry (CTA barrier above)
  }
  if (probe) {
    const long long cc = clock64();
    c_hand += cc - tc;
    prof[10] += (unsigned long long)c_hand;
    prof[11] += (unsigned long long)c_mv;
  }
  R.head = b;
  ring = R;
  return ok;
}

}  // namespace spock
