// spock_dev.cuh -- device-side building blocks of libspock (sm_103a).
//
// Problem descriptor handed to every kernel, team-level (1..8 warps) mat-vecs
// over per-node matrices stored "input-major" (row k = input index, columns =
// outputs, leading dimension padded to 4 elements so rows are 16-byte
// aligned), warp/block reductions with a fixed order (bit-reproducible), and
// a grid barrier with a time limit that reports an error instead of hanging.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spock {

constexpr int MAXD = 256;          // max nx + nu
constexpr int MAXTW = 8;           // max warps per team
constexpr int NRED = 8;            // reduction slots per T evaluation

// ---------------------------------------------------------------------------
// Problem descriptor (all pointers device, T = float or double)
// ---------------------------------------------------------------------------
template <class T>
struct Prob {
  // sizes
  int n, n_nl, n_l, N, nx, nu, n_c, n_cN, nbx, nbu, nbox, has_ball;
  long long nz, neta, nv;
  // z layout
  long long o_x, o_u, o_y, o_tau, o_s;
  // eta layout (relative to the start of eta)
  long long e_y, e_s, e_c, e_q, e_cN, e_qN;
  int W;                       // nx + nu + 2 (cost block of a non-root node)
  int ldB, ldF, ldP, ldK;      // leading dims of MB, MF, MP, KT
  // tree (breadth-first, children contiguous)
  const int* anc;              // [n]
  const int* ch_off;           // [n_nl + 1]
  const int* yoff;             // [n_nl + 1]
  // schedule of the sweeps: chains of single-child non-leaf nodes ("segments")
  int n_levels;
  const int* lvl_off;          // [n_levels + 1] into the segment arrays (bottom-up order)
  const int* seg_top;          // top node of a segment
  const int* seg_bot;          // bottom node
  const int* seg_len;          // number of nodes
  const int* seg_off;          // start of the segment's node list in seg_nodes
  const int* seg_nodes;        // nodes of every segment, top to bottom, contiguous
  const int4* seg_info;        // per segment: (list offset, length, first and one-past-last
                               // child of the bottom node)
  // per-iteration factors (built offline in FP64 from Alg. 1)
  const T* MB;   // per non-root c: [Abar_c | B_c Rt^{-1}]      nx x ldB   (input: q_c + P_c c_c)
  const T* MF;   // per non-root c: [Abar_c^T ; B_c^T]           (nx+nu) x ldF (input: [x; d])
  const T* MP;   // per non-leaf i: [K_i | Rt_i^{-1}]             nu x ldP   (input: ubar)
  const T* KT;   // per non-leaf i: K_i^T                        nx x ldK   (input: x)
  const T* cvec; // per non-root: scaled c (nx)
  const T* kc;   // per non-leaf i: sum_c MB_c' (P_c c_c) (nx + nu), the constant part of
                 // the backward recursion added to h^i and subtracted from e^i
  int pipe_bytes;  // largest per-node matrix in bytes when it is streamed through
                   // shared memory (0: matrices read from global memory)
  // whole-CTA sweeps (cta = 1, nx + nu <= 128): the factors stored
  // output-column-major, the coefficients of one output column contiguous
  int cta;
  int ldTB, ldTF, ldTK;  // padded length of one column of MBt (nx), MFt (nx+nu), KTt (nx)
  int khB, khF;          // first row of the second thread of a column (nx rows / nx+nu rows)
  int nbuf;              // depth of the ring of item buffers (2..4)
  int item_bytes;        // bytes of one ring buffer (multiple of 128)
  int qslots;            // child inputs of a backward bottom held at once
  int ldc;               // elements of one carry or child-input vector
  const int* top_seg;  // [n] segment whose top node is i, or -1
  const int* bot_seg;  // [n] segment whose bottom node is i, or -1
  int seg_flag_off;    // segment flags start at flags + seg_flag_off (after the barrier flags)
  const T* MBt;  // per non-root c: (nx+nu) columns x ldTB  (MB transposed)
  const T* MFt;  // per non-root c: nx columns x ldTF       (MF transposed)
  const T* KTt;  // per non-leaf i: nu columns x ldTK       (KT transposed)
  // cost and constraint data (scaled, Sec. 5.4)
  const T* qh;   // per non-root: diag of Q^{1/2} S^{-1} (nx)
  const T* rh;   // per non-root: diag of R^{1/2} Su^{-1} (nu)
  const T* qNh;  // per leaf (nx)
  const T* gx;   // nx: coefficient of the x-box rows
  const T* gu;   // nu: coefficient of the u-box and u-ball rows
  const T* gN;   // nx: coefficient of the leaf x-box rows
  const T* box_lo; const T* box_hi;    // [n_nl nbox]
  const T* boxN_lo; const T* boxN_hi;  // [n_l nx]
  const T* ball;                       // [n_nl]
  const T* prob;                       // [n] conditional probabilities
  const T* avar;                       // [n_nl]
  const T* x0s;                        // [nx] scaled initial state
  // full weights (full = 1): scaled upper Cholesky factors F S^{-1} of every
  // Q^c, R^c (non-root c) and Q_N^j (leaf j), row-major, and their transposes
  int full;
  const T *FQ, *FQT;   // [(n-1) nx nx]
  const T *FR, *FRT;   // [(n-1) nu nu]
  const T *FN, *FNT;   // [n_l nx nx]
  // translation of each cost cone (Prop. 1 with linear terms), or null for
  // (0, .., 1/2, -1/2): per non-root node W entries, per leaf nx + 2
  const T* acost;
  const T* acostN;
  // general constraint rows (scaled, Sec. 5.4): n_g rows G = [Gx Gu] at every
  // non-leaf node after the box and ball rows, n_gN rows GN at every leaf after
  // the x box rows; the sets are boxes per node
  int n_g, n_gN;
  const T* Gg;         // [n_g (nx + nu)]
  const T* GgT;        // [(nx + nu) n_g]
  const T* GgN;        // [n_gN nx]
  const T* GgNT;       // [nx n_gN]
  const T *gen_lo, *gen_hi;     // [n_nl n_g]
  const T *genN_lo, *genN_hi;   // [n_l n_gN]
  T alpha;
  // Centred form (FP32 iteration about an FP64 centre c = (z_c, eta_c)): the
  // kernel then evaluates D(delta) = T(c + delta) - c. lin = 1 drops the
  // constant terms of prox_f (x0s, cvec and kc then point at zeros); cz = z+_c
  // - z_c is added to every z output (and taken off again where a sweep reads
  // back an x it wrote); the eta prox steps run in FP64 on the full argument,
  // with ctrA = (eta_c + alpha L z_c)/alpha - a and ctrB = alpha L z_c - alpha a
  // per element of eta (a: the translation of the element's set, zero outside
  // the cost cones). Null / zero in the plain form.
  int lin;
  const T* cz;                 // [nz]
  const double* ctrA;          // [neta]
  const double* ctrB;          // [neta]
  double ctr_al, ctr_ial;      // alpha and 1/alpha in FP64
  // scratch of the sweeps
  T* qbuf;   // [n nx]
  T* dbuf;   // [n_nl nu]
  T* hbuf;   // [n_nl nx]   -K'ubar - xbar
  T* ebuf;   // [n_nl nu]   Rt^{-1} ubar
  // l1 edge-cost term lambda_0 ||(x^anc, u^anc)||_1 (Prop. 2; l1 = lambda_0,
  // 0 = none): theta^i at o_th + i and lambda^i (scaled like (x^i, u^i)) at
  // o_lam + i (nx + nu) in z; per non-leaf node the rows theta - sum_k l1w_k
  // lambda_k, lambda - (x^i, u^i), lambda + (x^i, u^i), all in R_+, at
  // e_l1 + i (1 + 2 (nx + nu)) in eta; the cost cone of every child c of i
  // carries (tau^c - l1 theta^i)/2 in its last two entries.
  // Risk of the non-leaf nodes (Sec. 3.3): tv = 0: AV@R with the levels in
  // avar, y^i = 2 m + 1 entries, b = [p; 0; 1]; tv = 1: the total-variation
  // ball of radius tvr[i], y^i = 3 m + 2 entries [y1 | y2 | y3 | y4 | y5] (m, m,
  // 1, m, 1), b = [p; -p; r; 0; 1], every entry but the last in R_+.
  int tv;
  const T* tvr;
  // soft-constraint costs ||max(0, (x^anc, u^anc) - z_max)||^2 (after Prop. 2;
  // soft = 0: none): sigma^i at o_sg + i and theta^i (scaled like (x^i, u^i))
  // at o_sth + i (nx + nu) in z; per non-leaf node at e_sf + i (3 d + 2), d =
  // nx + nu, the rows [smw theta, sigma/2, sigma/2] in SOC_{d+2} + (0, 1/2,
  // -1/2), theta in R_+^d, theta - (x^i, u^i) >= slo; the cost cone of every
  // child c of i carries (tau^c - sigma^i)/2 in its last two entries.
  int soft;
  long long o_sg, o_sth, e_sf;
  const T* smw;   // [d] 1/S^x, 1/S^u
  const T* slo;   // [d] -S^x z_max, -S^u z_max
  T l1;
  long long o_th, o_lam, e_l1;
  const T* l1w;   // [nx + nu] 1/S^x, 1/S^u
  // Mailboxes of the whole-CTA sweeps, n (nx + nu) values each, every 32-bit
  // piece of a value stored in one 64-bit word beside a 32-bit tag (the
  // evaluation's sweep epoch), so that a reader knows from the word itself
  // that it is current: mbb[top] holds a segment top's share of its parent's
  // backward step, mbf[bottom] the [x; d] of a segment bottom for the
  // segments of its children. Zeroed before every launch.
  unsigned long long* mbb;
  unsigned long long* mbf;
};

// Bounds-checked build (-DSPOCK_CHECKED, libspock_checked.so): the indices
// the iteration kernel derives from the tree (children, segment nodes,
// mailbox slots, the factors a bulk copy reads) are checked before use. A
// failing check records its site in the launch's control block, raises the
// launch's error word (every CTA then leaves at its next wait) and skips the
// access; nothing traps. Compiled out otherwise (SPOCK_CHK is true). One
// launch at a time: the kernel publishes the control block through a
// per-module global at entry.
#ifdef SPOCK_CHECKED
__device__ int* g_chk_err;
__device__ int* g_chk_site;
__device__ __forceinline__ bool chk_index(bool ok, int site) {
  if (!ok && g_chk_err) {
    atomicCAS(g_chk_site, 0, site);
    atomicExch(g_chk_err, 3);
  }
  return ok;
}
#define SPOCK_CHK(ok, site) ::spock::chk_index((ok), (site))
#else
#define SPOCK_CHK(ok, site) true
#endif

// entry k of b^i (conic risk data of node i with m children, first child c0)
template <class T>
__device__ __forceinline__ T risk_b(const Prob<T>& P, int i, int c0, int m, int k) {
  if (!P.tv) return (k < m) ? P.prob[c0 + k] : (k == 2 * m ? T(1) : T(0));
  if (k < m) return P.prob[c0 + k];
  if (k < 2 * m) return -P.prob[c0 + k - m];
  if (k == 2 * m) return P.tvr[i];
  return (k == 3 * m + 1) ? T(1) : T(0);
}
// entries of y^i in R_+ (the rest, the last entry, is free: the zero cone's dual)
template <class T>
__device__ __forceinline__ int risk_npos(const Prob<T>& P, int m) {
  return P.tv ? 3 * m + 1 : 2 * m;
}

// ---------------------------------------------------------------------------
// memory helpers: data written inside a kernel is read through L2 (ld.cg) so a
// stale L1 line of an earlier phase is never used; read-only data uses ldg.
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T ldc(const T* p) { return __ldcg(p); }
template <class T> __device__ __forceinline__ void stc(T* p, T v) { __stcg(p, v); }
template <class T> __device__ __forceinline__ T ldr(const T* p) { return __ldg(p); }

// z output of element idx: in the centred form the linear part plus cz
template <class T>
__device__ __forceinline__ T zc_add(const Prob<T>& P, long long idx, T v) {
  return P.cz ? v + ldr(P.cz + idx) : v;
}
// the linear part of an x the sweep wrote (centred form: minus cz)
template <class T>
__device__ __forceinline__ T zc_sub(const Prob<T>& P, long long idx, T v) {
  return P.cz ? v - ldr(P.cz + idx) : v;
}

template <class T> struct Vec;
template <> struct Vec<float> { using V = float4; static constexpr int N = 4; };
template <> struct Vec<double> { using V = double2; static constexpr int N = 2; };

template <class T>
__device__ __forceinline__ void vload(const T* p, T (&o)[Vec<T>::N]);
template <>
__device__ __forceinline__ void vload<float>(const float* p, float (&o)[4]) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void vload<double>(const double* p, double (&o)[2]) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  o[0] = v.x; o[1] = v.y;
}

// ---------------------------------------------------------------------------
// team = tw consecutive warps of a CTA; synchronised by a named barrier
// ---------------------------------------------------------------------------
struct Team {
  int tw, id, warp, lane, tid, nth;
  __device__ __forceinline__ void sync() const {
    if (tw == 1) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(nth) : "memory");
    }
  }
};

__device__ __forceinline__ Team make_team(int tw) {
  Team t;
  const int w = threadIdx.x >> 5;
  t.tw = tw;
  t.id = w / tw;
  t.warp = w % tw;
  t.lane = threadIdx.x & 31;
  t.tid = t.warp * 32 + t.lane;
  t.nth = tw * 32;
  return t;
}

// Register accumulator of one lane for a team mat-vec: the lane owns column
// chunks (c*32 + lane)*VEC .. +VEC, c < CH; the widest output is D = 32*VEC*CH.
template <class T, int CH>
struct Acc {
  static constexpr int VEC = Vec<T>::N;
  static constexpr int D = 32 * VEC * CH;
  T a[CH][VEC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int e = 0; e < VEC; ++e) a[c][e] = T(0);
  }
};

// acc += sum_k M[k*ld + j] * in[k] for j < ncols, k < nrows. Rows are split
// over the team's warps (warp w takes rows w, w+tw, ...), columns over lanes.
// Loads of RB rows are issued before their FMAs so a warp has RB*CH 16-byte
// loads in flight.
template <class T>
__device__ __forceinline__ void vload_s(const T* p, T (&o)[Vec<T>::N]);
template <>
__device__ __forceinline__ void vload_s<float>(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void vload_s<double>(const double* p, double (&o)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x; o[1] = v.y;
}

// SMEM = true: M lives in shared memory (filled by a bulk copy); false: M is
// read-only global memory read through the non-coherent path.
template <class T, int CH, bool SMEM = false>
__device__ __forceinline__ void team_mv(const Team& tm, Acc<T, CH>& acc, const T* __restrict__ M,
                                        int ld, int nrows, int ncols, const T* in) {
  constexpr int VEC = Vec<T>::N;
  constexpr int RB = (sizeof(T) == 4) ? 8 : 4;
  const int step = tm.tw;
  for (int k0 = tm.warp; k0 < nrows; k0 += RB * step) {
    T m[RB][CH][VEC];
    T xk[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int k = k0 + r * step;
      const bool okr = k < nrows;
      xk[r] = okr ? in[k] : T(0);
      const T* row = M + (size_t)(okr ? k : 0) * ld;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int col = (c * 32 + tm.lane) * VEC;
        if (okr && col < ncols) {
          if (SMEM) vload_s<T>(row + col, m[r][c]);
          else vload<T>(row + col, m[r][c]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) m[r][c][e] = T(0);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc.a[c][e] = fma(m[r][c][e], xk[r], acc.a[c][e]);
  }
}

// Sum the warps' accumulators (fixed order) and call f(j, m, value) for every
// output j < ncols owned by this thread (j = tid + m*nth, m a compile-time
// index so per-thread register arrays can be indexed by it). red: team
// scratch of tw*D elements. Ends with a team sync.
template <class T, int CH, class F>
__device__ __forceinline__ void team_reduce(const Team& tm, const Acc<T, CH>& acc, int ncols,
                                            T* red, F&& f) {
  constexpr int VEC = Vec<T>::N;
  constexpr int D = Acc<T, CH>::D;
  constexpr int PT = D / 32;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = (c * 32 + tm.lane) * VEC;
    if (col < ncols) {
#pragma unroll
      for (int e = 0; e < VEC; ++e)
        if (col + e < ncols) red[tm.warp * D + col + e] = acc.a[c][e];
    }
  }
  tm.sync();
#pragma unroll
  for (int m = 0; m < PT; ++m) {
    const int j = tm.tid + m * tm.nth;
    if (j < ncols) {
      T s = red[j];
      for (int w = 1; w < tm.tw; ++w) s += red[w * D + j];
      f(j, m, s);
    }
  }
  tm.sync();
}

// ---------------------------------------------------------------------------
// warp reductions (fixed butterfly order)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-thread partial sums of one T evaluation (see RedIdx).
enum RedIdx {
  R_MAX = 0,     // max |r|
  R_ZZ = 1,      // ||r_z||^2
  R_EE = 2,      // ||r_eta||^2
  R_ELZ = 3,     // <r_eta, L r_z>
  R_ZD = 4,      // <r_z, dz>       (dz = z_in - z_ref)
  R_ED = 5,      // <r_eta, deta>
  R_LZD = 6,     // <L r_z, deta>
  R_ELD = 7      // <r_eta, L dz>
};

template <class T>
struct RedAcc {
  T v[NRED];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NRED; ++i) v[i] = T(0);
  }
  // z element: old value, new value, direction value (0 when absent)
  __device__ __forceinline__ void z(T old, T nw, T dir) {
    const T r = old - nw;
    v[R_MAX] = max(v[R_MAX], fabs(r));
    v[R_ZZ] = fma(r, r, v[R_ZZ]);
    v[R_ZD] = fma(r, dir, v[R_ZD]);
  }
  // eta element: old and new eta values, the direction's eta value ed,
  // lrz = L(z_old - z_new) and lod = L(d_z) of the element's row. L is applied
  // to the differences (not differences of L applied: near convergence z_old
  // and z_new agree to many digits and the difference of two rounded products
  // would be noise), and the direction d is read as stored instead of being
  // recovered as v~ - v.
  __device__ __forceinline__ void eta(T eo, T en, T ed, T lrz, T lod) {
    const T r = eo - en;
    v[R_MAX] = max(v[R_MAX], fabs(r));
    v[R_EE] = fma(r, r, v[R_EE]);
    v[R_ELZ] = fma(r, lrz, v[R_ELZ]);
    v[R_ED] = fma(r, ed, v[R_ED]);
    v[R_LZD] = fma(lrz, ed, v[R_LZD]);
    v[R_ELD] = fma(r, lod, v[R_ELD]);
  }
};

// Combine step of the NRED-value reductions: the sum, or for the max slot the
// maximum taken on the bit patterns (which order non-negative doubles like
// their values; a NaN wins, so a NaN residual never reads as converged).
__device__ __forceinline__ double red_comb(double a, double b, bool is_max) {
  const long long m = max(__double_as_longlong(a), __double_as_longlong(b));
  return is_max ? __longlong_as_double(m) : a + b;
}

// Warp reduction of NRED = 8 doubles in 9 FP64 additions per lane instead of
// 8 x 5: each butterfly step sends half of the values a lane still carries to
// its partner, so after three steps a lane carries one value and two more
// steps finish it. On return lane l holds the warp total of value
// 4 b4 + 2 b3 + b2 (b = the bits of l); lane 4k holds value k. FP64 runs at a
// small fraction of the FP32 rate on this part, so the count matters.
__device__ __forceinline__ double warp_reduce8(const double (&v)[NRED], int max_slot) {
  static_assert(NRED == 8, "warp_reduce8 is written for 8 values");
  const int lane = threadIdx.x & 31;
  const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0, h2 = (lane & 4) != 0;
  double u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double keep = h4 ? v[4 + j] : v[j];
    const double send = h4 ? v[j] : v[4 + j];
    u[j] = red_comb(keep, __shfl_xor_sync(0xffffffffu, send, 16), (h4 ? 4 : 0) + j == max_slot);
  }
  double w[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double keep = h3 ? u[2 + j] : u[j];
    const double send = h3 ? u[j] : u[2 + j];
    w[j] = red_comb(keep, __shfl_xor_sync(0xffffffffu, send, 8), (h4 ? 4 : 0) + (h3 ? 2 : 0) + j == max_slot);
  }
  const bool mx = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0) == max_slot;
  double x = red_comb(h2 ? w[1] : w[0], __shfl_xor_sync(0xffffffffu, h2 ? w[0] : w[1], 4), mx);
  x = red_comb(x, __shfl_xor_sync(0xffffffffu, x, 2), mx);
  x = red_comb(x, __shfl_xor_sync(0xffffffffu, x, 1), mx);
  return x;
}

// Block reduction of NRED doubles: on return every thread's v[] holds the
// block totals. Slot `max_slot` takes the maximum (-1: none; its values must
// be non-negative), the others the sum, in a fixed order.
// scratch: NRED * 32 doubles of shared memory.
__device__ __forceinline__ void block_reduce_red(double (&v)[NRED], double* scratch, int max_slot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double x = warp_reduce8(v, max_slot);
  if ((lane & 3) == 0) scratch[(lane >> 2) * 32 + w] = x;
  __syncthreads();
  if (w == 0 && lane < NRED) {   // lane k adds the warps' totals of value k
    double t = scratch[lane * 32];
    for (int j = 1; j < nw; ++j) t = red_comb(t, scratch[lane * 32 + j], lane == max_slot);
    scratch[lane * 32] = t;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NRED; ++i) v[i] = scratch[i * 32];
  __syncthreads();   // the next call may overwrite scratch
}

// ---------------------------------------------------------------------------
// grid barrier with a time limit. `count` counts arrivals for the whole launch
// (never reset), so barrier number e completes when count reaches e*gridDim.x;
// the last CTA to arrive may run a callback (whole CTA) and then publishes
// `gen` = e with a release store, which the others wait for. On timeout the
// error word is set and every CTA leaves at its next check.
// ---------------------------------------------------------------------------
struct GridCtl {
  unsigned int count;
  unsigned int gen;
  int error;          // 0 ok, else a timeout happened
  int pad;
};

// The group of CTAs that iterates on one problem: the whole grid (one problem
// per launch), or one CTA (local = true: the batched launch, where every CTA
// works on its own problem and the barriers and reductions stay in the CTA).
struct Grid {
  GridCtl* ctl;       // error word
  unsigned* flags;    // one arrival flag per CTA of the group (zeroed before the launch)
  double* partials;   // 2 x size x NRED reduction partials (double-buffered)
  unsigned epoch;     // barriers passed by this CTA (identical on every CTA)
  unsigned long long* prof;   // cycle counters of CTA 0 (slots 12..15), may be null
  int rank, size;     // this CTA's index in the group and the group's size
  bool local;
  uint64_t limit_ns;  // give up a barrier wait after this long
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_i(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr uint64_t BARRIER_LIMIT_NS = 2000000000ull;   // 2 s per wait

// Flag barrier: CTA b publishes flags[b] = epoch with a release store (after a
// CTA barrier, so the release covers every thread's earlier writes); thread t
// then waits with acquire loads until flags[t], flags[t + blockDim], ... reach
// the epoch. No atomics and no central counter: two L2 round trips.
// Returns false when the launch is in error (timeout here or elsewhere).
__device__ __forceinline__ bool poll_flags(Grid& g, unsigned e) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < g.size; c += blockDim.x) {
    uint64_t t0 = 0;
    unsigned spins = 0;
    while (ld_acquire(g.flags + c) < e) {
      __nanosleep(64);   // back off: idle CTAs must not flood L2 while others work
      if ((++spins & 63u) == 0u) {
        if (ld_relaxed_i(&g.ctl->error)) { s_bad = 1; break; }
        const uint64_t t = global_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > g.limit_ns) {
          atomicExch(&g.ctl->error, 1);
          s_bad = 1;
          break;
        }
      }
    }
  }
  __syncthreads();
  return s_bad == 0;
}

__device__ __forceinline__ bool grid_sync(Grid& g) {
  if (g.local) {
    __syncthreads();
    return true;
  }
  const bool probe = g.prof && blockIdx.x == 0 && threadIdx.x == 0;
  const long long t0 = probe ? clock64() : 0;
  const unsigned e = ++g.epoch;
  __syncthreads();
  if (threadIdx.x == 0) st_release(g.flags + g.rank, e);
  const bool ok = poll_flags(g, e);
  if (probe) {
    g.prof[12] += (unsigned long long)(clock64() - t0);
    g.prof[14] += 1;
  }
  return ok;
}

// All-reduce of NRED doubles over the grid: slot max_slot by max (-1: none),
// the others by sum. Every CTA combines the per-CTA partials in the same
// fixed order, so every CTA gets bit-identical results. scratch: shared
// memory of NRED * 32 doubles. Returns false on error.
__device__ __forceinline__ bool grid_allreduce(Grid& g, double (&v)[NRED], double* scratch,
                                               int max_slot) {
  if (g.local) {
    block_reduce_red(v, scratch, max_slot);
    return true;
  }
  const bool probe = g.prof && blockIdx.x == 0 && threadIdx.x == 0;
  const long long t0 = probe ? clock64() : 0;
  block_reduce_red(v, scratch, max_slot);
  const unsigned e = ++g.epoch;
  double* part = g.partials + (size_t)(e & 1u) * g.size * NRED;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NRED; ++k) __stcg(part + (size_t)g.rank * NRED + k, v[k]);
    st_release(g.flags + g.rank, e);
  }
  const bool ok = poll_flags(g, e);
  double x[NRED];
#pragma unroll
  for (int k = 0; k < NRED; ++k) x[k] = 0.0;
  for (int c = threadIdx.x; c < g.size; c += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
      const double y = __ldcg(part + (size_t)c * NRED + k);
      x[k] = red_comb(x[k], y, k == max_slot);
    }
  }
  block_reduce_red(x, scratch, max_slot);
#pragma unroll
  for (int k = 0; k < NRED; ++k) v[k] = x[k];
  if (probe) {
    g.prof[13] += (unsigned long long)(clock64() - t0);
    g.prof[15] += 1;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// The same reductions on float pairs for the FP32 kernels. A pair (h, l)
// stands for h + l (double-float); the FP32 partials enter as (v, 0), a
// compensated sum as (sum, error). FP64 issues at about 1/77 of the FP32 rate
// on this part, and the FP64 warp, CTA and grid combines above cost several
// thousand cycles per all-reduce; these run on the FP32 pipe. A sum step is an
// error-free two-sum of the high parts (Knuth's TwoSum) with the low parts
// added to its error term and the result renormalised by a fast two-sum
// (Dekker): relative error about 2^-44 of the summands' magnitudes, far below
// the FP32 partials' own. The max slot takes the maximum of the high parts'
// bit patterns (non-negative values; a NaN wins). Fixed order throughout, so
// every CTA gets bit-identical results; they are returned as doubles (h + l,
// exact in FP64).
// ---------------------------------------------------------------------------
struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_comb(DF a, DF b, bool is_max) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  const float t = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, t);
  const DF sum{h, __fsub_rn(t, __fsub_rn(h, s))};
  const DF mx{__int_as_float(max(__float_as_int(a.h), __float_as_int(b.h))), 0.0f};
  return is_max ? mx : sum;
}

__device__ __forceinline__ DF df_shfl_xor(DF a, int m) {
  return DF{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
}

// warp_reduce8 on pairs: the same butterfly, the same lane holding each total.
__device__ __forceinline__ DF warp_reduce8_df(const DF (&v)[NRED], int max_slot) {
  static_assert(NRED == 8, "warp_reduce8_df is written for 8 values");
  const int lane = threadIdx.x & 31;
  const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0, h2 = (lane & 4) != 0;
  DF u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const DF keep = h4 ? v[4 + j] : v[j];
    const DF send = h4 ? v[j] : v[4 + j];
    u[j] = df_comb(keep, df_shfl_xor(send, 16), (h4 ? 4 : 0) + j == max_slot);
  }
  DF w[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const DF keep = h3 ? u[2 + j] : u[j];
    const DF send = h3 ? u[j] : u[2 + j];
    w[j] = df_comb(keep, df_shfl_xor(send, 8), (h4 ? 4 : 0) + (h3 ? 2 : 0) + j == max_slot);
  }
  const bool mx = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0) == max_slot;
  DF x = df_comb(h2 ? w[1] : w[0], df_shfl_xor(h2 ? w[0] : w[1], 4), mx);
  x = df_comb(x, df_shfl_xor(x, 2), mx);
  x = df_comb(x, df_shfl_xor(x, 1), mx);
  return x;
}

// CTA totals of NRED pairs: on return (after a CTA barrier) scratch[k * 32]
// holds the total of value k. scratch: NRED * 32 pairs of shared memory.
__device__ __forceinline__ void block_reduce_df(const DF (&v)[NRED], DF* scratch, int max_slot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const DF x = warp_reduce8_df(v, max_slot);
  if ((lane & 3) == 0) scratch[(lane >> 2) * 32 + w] = x;
  __syncthreads();
  if (w == 0 && lane < NRED) {   // lane k adds the warps' totals of value k
    DF t = scratch[lane * 32];
    for (int j = 1; j < nw; ++j) t = df_comb(t, scratch[lane * 32 + j], lane == max_slot);
    scratch[lane * 32] = t;
  }
  __syncthreads();
}

// grid_allreduce on pairs: out[k] (every thread) = the grid total of value k
// as a double. scratch: NRED * 32 pairs, tot: NRED doubles, both shared.
__device__ __forceinline__ bool grid_allreduce_df(Grid& g, const DF (&v)[NRED], double (&out)[NRED], DF* scratch,
                                                  double* tot, int max_slot) {
  const bool probe = !g.local && g.prof && blockIdx.x == 0 && threadIdx.x == 0;
  const long long t0 = probe ? clock64() : 0;
  block_reduce_df(v, scratch, max_slot);
  bool ok = true;
  if (!g.local) {
    const unsigned e = ++g.epoch;
    float2* part = reinterpret_cast<float2*>(g.partials) + (size_t)(e & 1u) * g.size * NRED;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < NRED; ++k) {
        const DF t = scratch[k * 32];
        __stcg(part + (size_t)g.rank * NRED + k, make_float2(t.h, t.l));
      }
      st_release(g.flags + g.rank, e);
    }
    ok = poll_flags(g, e);
    DF x[NRED];
#pragma unroll
    for (int k = 0; k < NRED; ++k) x[k] = DF{0.0f, 0.0f};
    for (int c = threadIdx.x; c < g.size; c += blockDim.x) {
#pragma unroll
      for (int k = 0; k < NRED; ++k) {
        const float2 y = __ldcg(part + (size_t)c * NRED + k);
        x[k] = df_comb(x[k], DF{y.x, y.y}, k == max_slot);
      }
    }
    block_reduce_df(x, scratch, max_slot);
  }
  if (threadIdx.x < NRED) {
    const DF t = scratch[threadIdx.x * 32];
    tot[threadIdx.x] = (double)t.h + (double)t.l;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NRED; ++k) out[k] = tot[k];
  __syncthreads();   // the next call may overwrite scratch and tot
  if (probe) {
    g.prof[13] += (unsigned long long)(clock64() - t0);
    g.prof[15] += 1;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (cp.async.bulk, global -> shared) with a bounded wait
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the mbarrier; false (and *err set) after the
// time limit. A second bounded wait lets a late copy land before the caller
// leaves, so no copy into this CTA's shared memory is left in flight.
// diag (may be null): 4 ints recording the first wait that gave up
// (CTA, buffer address, parity, site)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err,
                                          int* diag = nullptr, int site = 0) {
  unsigned spins = 0;
  uint64_t t0 = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 255u) == 0u) {
      if (ld_relaxed_i(err)) return false;      // the launch is already failing: leave now
      const uint64_t t = global_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > BARRIER_LIMIT_NS) {
        if (atomicCAS(err, 0, 2) == 0 && diag) {
          diag[0] = blockIdx.x;
          diag[1] = (int)smem_u32(bar);
          diag[2] = (int)parity;
          diag[3] = site;
        }
        const uint64_t t1 = global_ns();
        while (!mbar_try_wait(bar, parity) && global_ns() - t1 < BARRIER_LIMIT_NS) {
        }
        return false;
      }
    }
  }
  return true;
}

// Double-buffered stream of per-node matrices into a team's shared memory.
// Thread 0 of the team issues the copies; every thread waits. par[] keeps the
// phase of each buffer's mbarrier for the whole launch.
template <class T>
struct Pipe {
  uint64_t* bar;     // 2 mbarriers
  T* buf[2];
  unsigned par[2];
  int cur;
  bool on;           // false: matrices are read from global memory
  int* okp;          // shared int of the team: result of the last wait
  int* diag;         // where the first wait that gave up is recorded
  __device__ __forceinline__ void issue(const Team& tm, int b, const T* src, unsigned bytes) {
    if (tm.tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar + b, bytes);
      bulk_g2s(buf[b], src, bytes, bar + b);
    }
  }
  // thread 0 of the team polls the mbarrier (non-suspending test_wait); the
  // team barrier then hands the completed copy to every thread of the team
  // ok_slot: shared int of this team that hands the result to every thread
  __device__ __forceinline__ bool wait(const Team& tm, int b, int* err, int* ok_slot,
                                       int* diag = nullptr, int site = 0) {
    if (tm.tid == 0) *ok_slot = mbar_wait(bar + b, par[b], err, diag, site) ? 1 : 0;
    par[b] ^= 1u;
    tm.sync();
    return *ok_slot != 0;
  }
};

}  // namespace spock
