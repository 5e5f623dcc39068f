// spock_solver_kernel.cuh -- the SPOCK iteration as one persistent cooperative kernel.
//
// One evaluation of the Chambolle-Pock operator T (Eq. chambolle-pock-operator)
// is four phases. Grid barriers follow P and F, and an all-reduce ends E; the
// tree levels inside B and F are ordered by per-segment flags in the
// whole-CTA sweeps (spock_cta.cuh) and by a barrier per level in the team
// sweeps:
//
//  P (one warp per node): w = z - alpha L* eta for the node's own blocks
//    (sibling sums of L* read the children's cost blocks), the s0 update
//    (prox of f's linear term), the S2 projection of (y^i, tau^[i], s^[i]) in
//    closed form (Sherman-Morrison on GG' = (a^2+3) I + 11'), and the parts of
//    Alg. 2 that do not depend on the sweep:
//      h^i = -K_i' ubar^i - xbar^i,  e^i = Rt_i^{-1} ubar^i,  q^leaf = -xbar.
//  B (backward sweep of Alg. 2, bottom-up over "segments" = chains of
//    single-child non-leaf nodes, which a team walks without a grid barrier,
//    carrying q down the chain in shared memory):
//      v_c = q_c + P_c c_c;  q^i = sum_c Abar_c' v_c + h^i;
//      d^i = e^i - sum_c (B_c Rt_i^{-1})' v_c.
//    (Alg. 2's qbar holds the extra term (K' + sum Abar'PB) d, which is zero
//    because K = -Rt^{-1} sum B'PA; the kernel uses the reduced form.)
//  F (forward rollout of Alg. 2, top-down over segments):
//      u^i = K x^i + d^i,  x^c = Abar_c x^i + B_c d^i + c_c.
//  E (one warp per block of eta): eta+ = prox_{alpha g*}(eta + alpha L(2z+ - z))
//    with the S3 projections (cones, boxes, ball, translated SOCs).
// Every phase also accumulates the reductions of r = v - T(v): max|r|,
// ||r_z||^2, ||r_eta||^2, <r_eta, L r_z>, and the M-inner product with a
// direction (the SuperMann candidate's psi); they are combined by one group
// reduction at the end.
//
// The SuperMann driver (Alg. 4) with Anderson directions (Alg. 3, m = 3) runs
// redundantly on every CTA from the group-reduced scalars, so all CTAs take
// the same branch; there is no host round trip per iteration.
//
// Three kernels run that iteration: k_solve (one problem, the whole grid),
// k_batch (many problems: gangs of CTAs for large ones, single CTAs for the
// rest) and k_serve (requests claimed from a ring in mapped host memory).
#include <cuda_runtime.h>
#include <math.h>

#pragma once
#include "spock_dev.cuh"
#include "spock_internal.h"
#include "spock_cta.cuh"

namespace spock {

constexpr int AA_M = 3;
constexpr double C0 = 0.99, C1 = 0.99, C2 = 0.99, BETA = 0.5, SIGMA = 0.1, LAMBDA = 1.0;

template <class T>
__device__ __forceinline__ T dirv(const T* vdir, long long idx) {
  return vdir ? ldc(vdir + idx) : T(0);
}

// phase timer of CTA 0 (thread 0): adds the time since the last mark to slot
// k of a shared-memory array that is written to the control block at exit
struct PhaseClock {
  uint64_t t;
  bool on;
  unsigned long long* prof;
  __device__ __forceinline__ void start(unsigned long long* p) {
    prof = p;
    on = (blockIdx.x == 0 && threadIdx.x == 0);
    if (on) t = global_ns();
  }
  __device__ __forceinline__ void mark(SolveCtl*, int k) {
    if (on) {
      const uint64_t n = global_ns();
      prof[k] += n - t;
      t = n;
    }
  }
};

// ---------------------------------------------------------------------------
// Phase P
// ---------------------------------------------------------------------------
template <class T>
__device__ void s2_block(const Prob<T>& P, int lane, int i, const T* __restrict__ vin,
                         T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const int c0 = P.ch_off[i], m = P.ch_off[i + 1] - c0;
  if (!SPOCK_CHK(c0 >= 1 && m >= 1 && c0 + m <= P.n && P.yoff[i + 1] - P.yoff[i] == 2 * m + 1, 9)) return;
  const long long yo = P.o_y + P.yoff[i];
  const T al = P.alpha, a = P.avar[i];
  const T eS = ldc(eta + P.e_s + i);
  const T* ey = eta + P.e_y + P.yoff[i];
  auto wy = [&](int k) -> T {
    const T b = (k < m) ? P.prob[c0 + k] : (k == 2 * m ? T(1) : T(0));
    return ldc(z + yo + k) - al * (ldc(ey + k) - b * eS);
  };
  auto wt = [&](int l) -> T {
    const int c = c0 + l;
    const T* q = eta + P.e_q + (long long)(c - 1) * P.W;
    return ldc(z + P.o_tau + c - 1) - al * (T(0.5) * (ldc(q + nx + nu) + ldc(q + nx + nu + 1)));
  };
  auto ws = [&](int l) -> T {
    const int c = c0 + l;
    T g;
    if (c < P.n_nl) {
      g = ldc(eta + P.e_s + c);
    } else {
      const T* q = eta + P.e_qN + (long long)(c - P.n_nl) * (nx + 2);
      g = T(0.5) * (ldc(q + nx) + ldc(q + nx + 1));
    }
    return ldc(z + P.o_s + c - 1) - al * g;
  };
  const T y3 = wy(2 * m);
  T sg = 0;
  for (int l = lane; l < m; l += 32) sg += a * wy(l) - wy(m + l) + y3 - wt(l) - ws(l);
  sg = warp_sum(sg);
  const T cc = a * a + T(3);
  const T corr = sg / (cc + T(m));
  T sl = 0;
  for (int l = lane; l < m; l += 32) {
    const T wy1 = wy(l), wy2 = wy(m + l), wtl = wt(l), wsl = ws(l);
    const T gv = a * wy1 - wy2 + y3 - wtl - wsl;
    const T lam = (gv - corr) / cc;
    sl += lam;
    const int c = c0 + l;
    long long idx;
    idx = yo + l;           { const T o = ldc(z + idx), n1 = zc_add(P, idx, wy1 - a * lam); stc(vout + idx, n1); ra.z(o, n1, dirv(vref, idx)); }
    idx = yo + m + l;       { const T o = ldc(z + idx), n2 = zc_add(P, idx, wy2 + lam); stc(vout + idx, n2); ra.z(o, n2, dirv(vref, idx)); }
    idx = P.o_tau + c - 1;  { const T o = ldc(z + idx), nt = zc_add(P, idx, wtl + lam); stc(vout + idx, nt); ra.z(o, nt, dirv(vref, idx)); }
    idx = P.o_s + c - 1;    { const T o = ldc(z + idx), ns = zc_add(P, idx, wsl + lam); stc(vout + idx, ns); ra.z(o, ns, dirv(vref, idx)); }
  }
  sl = warp_sum(sl);
  if (lane == 0) {
    const long long idx = yo + 2 * m;
    const T n3 = zc_add(P, idx, y3 - sl);
    const T o = ldc(z + idx);
    stc(vout + idx, n3);
    ra.z(o, n3, dirv(vref, idx));
    if (i == 0) {   // s0 <- s0 - alpha (eta_s^0) - alpha (the last term is constant: not in the linear part)
      const T o0 = ldc(z);
      const T n0 = zc_add(P, 0, P.lin ? (o0 - al * eS) : (o0 - al * eS) - al);
      stc(vout, n0);
      ra.z(o0, n0, dirv(vref, 0));
    }
  }
}

// S2 with the total-variation risk (F != 0): projection of (y, tau^[i], s^[i])
// on ker G, G = [E', -I, -I; F', 0, 0], y = [y1 | y2 | y3 | y4 | y5]. E'E = 3I +
// 11', F'F = 2I + 11', E'F = 0, so GG' = blockdiag(5I + 11', 2I + 11') and
// both blocks invert in closed form (Sherman-Morrison):
//   g_E = y1 - y2 - y4 + y5 1 - tau - s,  g_F = -y1 - y2 + y3 1,
//   l_E = (g_E - 1 (1'g_E)/(5 + m))/5,   l_F = (g_F - 1 (1'g_F)/(2 + m))/2,
//   y1 -= l_E - l_F, y2 += l_E + l_F, y3 -= 1'l_F, y4 += l_E, y5 -= 1'l_E,
//   tau += l_E, s += l_E.
template <class T>
__device__ void s2_block_tv(const Prob<T>& P, int lane, int i, const T* __restrict__ vin,
                            T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const int c0 = P.ch_off[i], m = P.ch_off[i + 1] - c0;
  if (!SPOCK_CHK(c0 >= 1 && m >= 1 && c0 + m <= P.n && P.yoff[i + 1] - P.yoff[i] == 3 * m + 2, 9)) return;
  const long long yo = P.o_y + P.yoff[i];
  const T al = P.alpha;
  const T eS = ldc(eta + P.e_s + i);
  const T* ey = eta + P.e_y + P.yoff[i];
  auto wy = [&](int k) -> T { return ldc(z + yo + k) - al * (ldc(ey + k) - risk_b(P, i, c0, m, k) * eS); };
  auto wt = [&](int l) -> T {
    const T* q = eta + P.e_q + (long long)(c0 + l - 1) * P.W;
    T g = T(0.5) * (ldc(q + nx + nu) + ldc(q + nx + nu + 1));
    return ldc(z + P.o_tau + c0 + l - 1) - al * g;
  };
  auto ws = [&](int l) -> T {
    const int c = c0 + l;
    T g;
    if (c < P.n_nl) {
      g = ldc(eta + P.e_s + c);
    } else {
      const T* q = eta + P.e_qN + (long long)(c - P.n_nl) * (nx + 2);
      g = T(0.5) * (ldc(q + nx) + ldc(q + nx + 1));
    }
    return ldc(z + P.o_s + c - 1) - al * g;
  };
  const T y3 = wy(2 * m), y5 = wy(3 * m + 1);
  T sE = 0, sF = 0;
  for (int l = lane; l < m; l += 32) {
    const T y1 = wy(l), y2 = wy(m + l), y4 = wy(2 * m + 1 + l);
    sE += y1 - y2 - y4 + y5 - wt(l) - ws(l);
    sF += y3 - y1 - y2;
  }
  sE = warp_sum(sE);
  sF = warp_sum(sF);
  const T cE = sE / (T(5) + T(m)), cF = sF / (T(2) + T(m));
  T tE = 0, tF = 0;
  auto put = [&](long long idx, T val) {
    const T o = ldc(z + idx), nv = zc_add(P, idx, val);
    stc(vout + idx, nv);
    ra.z(o, nv, dirv(vref, idx));
  };
  for (int l = lane; l < m; l += 32) {
    const T y1 = wy(l), y2 = wy(m + l), y4 = wy(2 * m + 1 + l), wtl = wt(l), wsl = ws(l);
    const T lE = ((y1 - y2 - y4 + y5 - wtl - wsl) - cE) / T(5);
    const T lF = ((y3 - y1 - y2) - cF) / T(2);
    tE += lE;
    tF += lF;
    const int c = c0 + l;
    put(yo + l, y1 - lE + lF);
    put(yo + m + l, y2 + lE + lF);
    put(yo + 2 * m + 1 + l, y4 + lE);
    put(P.o_tau + c - 1, wtl + lE);
    put(P.o_s + c - 1, wsl + lE);
  }
  tE = warp_sum(tE);
  tF = warp_sum(tF);
  if (lane == 0) {
    put(yo + 2 * m, y3 - tF);
    put(yo + 3 * m + 1, y5 - tE);
    if (i == 0) {   // s0 <- s0 - alpha (eta_s^0) - alpha (the last term is constant: not in the linear part)
      const T o0 = ldc(z);
      const T n0 = zc_add(P, 0, P.lin ? (o0 - al * eS) : (o0 - al * eS) - al);
      stc(vout, n0);
      ra.z(o0, n0, dirv(vref, 0));
    }
  }
}

// The auxiliaries of the soft-constraint costs of node i: f does not involve
// them, so their step is w = z - alpha L*eta. L* of sigma^i: half the sum of
// the last two entries of its own cone minus the same of every child's cost
// cone; of theta^i_k: 1/s_k times its cone entry plus its rows theta >= 0 and
// theta - z >= lo.
template <class T>
__device__ void soft_prep(const Prob<T>& P, int lane, int i, const T* __restrict__ vin, T* __restrict__ vout,
                          const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu, d = nx + nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const T al = P.alpha;
  const T* es = eta + P.e_sf + (long long)i * (3 * d + 2);
  T sc = 0;
  for (int c = P.ch_off[i] + lane; c < P.ch_off[i + 1]; c += 32) {
    const T* eq = eta + P.e_q + (long long)(c - 1) * P.W + nx + nu;
    sc += ldc(eq) + ldc(eq + 1);
  }
  sc = warp_sum(sc);
  if (lane == 0) {
    const long long idx = P.o_sg + i;
    const T o = ldc(z + idx);
    const T n = zc_add(P, idx, o - al * (T(0.5) * (ldc(es + d) + ldc(es + d + 1)) - T(0.5) * sc));
    stc(vout + idx, n);
    ra.z(o, n, dirv(vref, idx));
  }
  for (int k = lane; k < d; k += 32) {
    const long long idx = P.o_sth + (long long)i * d + k;
    const T o = ldc(z + idx);
    const T n = zc_add(P, idx, o - al * (ldr(P.smw + k) * ldc(es + k) + ldc(es + d + 2 + k) + ldc(es + 2 * d + 2 + k)));
    stc(vout + idx, n);
    ra.z(o, n, dirv(vref, idx));
  }
}

// The auxiliaries of the l1 edge costs of node i (Prop. 2): f does not
// involve them, so their step is w = z - alpha L*eta. L* of theta^i: its l1
// row minus lambda_0/2 times the last two entries of every child's cost cone;
// of lambda^i_k: -w_k times the first l1 row plus the rows lambda_k - z_k and
// lambda_k + z_k.
template <class T>
__device__ void l1_prep(const Prob<T>& P, int lane, int i, const T* __restrict__ vin, T* __restrict__ vout,
                        const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu, d = nx + nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const T al = P.alpha;
  const T* el = eta + P.e_l1 + (long long)i * (1 + 2 * d);
  const T e0 = ldc(el);
  T sc = 0;
  for (int c = P.ch_off[i] + lane; c < P.ch_off[i + 1]; c += 32) {
    const T* eq = eta + P.e_q + (long long)(c - 1) * P.W + nx + nu;
    sc += ldc(eq) + ldc(eq + 1);
  }
  sc = warp_sum(sc);
  if (lane == 0) {
    const long long idx = P.o_th + i;
    const T o = ldc(z + idx);
    const T n = zc_add(P, idx, o - al * (e0 - T(0.5) * P.l1 * sc));
    stc(vout + idx, n);
    ra.z(o, n, dirv(vref, idx));
  }
  for (int k = lane; k < d; k += 32) {
    const long long idx = P.o_lam + (long long)i * d + k;
    const T o = ldc(z + idx);
    const T n = zc_add(P, idx, o - al * ((ldc(el + 1 + k) + ldc(el + 1 + d + k)) - ldr(P.l1w + k) * e0));
    stc(vout + idx, n);
    ra.z(o, n, dirv(vref, idx));
  }
}

// one warp (a team of one warp) per non-leaf node
template <class T, int CH>
__device__ void prep_nonleaf(const Prob<T>& P, const Team& tw1, T* s_in, T* s_xb, T* s_red, int i,
                             const T* __restrict__ vin, T* __restrict__ vout,
                             const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const int c0 = P.ch_off[i], c1 = P.ch_off[i + 1];
  if (!SPOCK_CHK(c0 >= 1 && c1 > c0 && c1 <= P.n, 10)) return;
  const T al = P.alpha;
  const T* ec = eta + P.e_c + (long long)i * P.n_c;
  const T* eg = ec + P.nbox + (P.has_ball ? nu : 0);   // general rows of node i
  for (int k = tw1.lane; k < nu; k += 32) {
    T g = 0;
    if (P.nbu) g += P.gu[k] * ldc(ec + P.nbx + k);
    if (P.has_ball) g += P.gu[k] * ldc(ec + P.nbox + k);
    for (int c = c0; c < c1; ++c) {
      const T* eq = eta + P.e_q + (long long)(c - 1) * P.W + nx;
      if (P.full) {   // (F_R^c)' eta_R^c
        const T* F = P.FR + (size_t)(c - 1) * nu * nu + k;
#pragma unroll 8
        for (int e = 0; e < nu; ++e) g = fma(ldr(F + (size_t)e * nu), ldc(eq + e), g);
      } else {
        g += ldr(P.rh + (long long)(c - 1) * nu + k) * ldc(eq + k);
      }
    }
#pragma unroll 8
    for (int r = 0; r < P.n_g; ++r) g = fma(ldr(P.GgT + (size_t)(nx + k) * P.n_g + r), ldc(eg + r), g);
    if (P.l1 != T(0)) {   // l1 rows lambda - u, lambda + u (Prop. 2)
      const T* el = eta + P.e_l1 + (long long)i * (1 + 2 * (nx + nu));
      g += ldc(el + 1 + (nx + nu) + nx + k) - ldc(el + 1 + nx + k);
    }
    if (P.soft) g -= ldc(eta + P.e_sf + (long long)i * (3 * (nx + nu) + 2) + 2 * (nx + nu) + 2 + nx + k);
    s_in[k] = ldc(z + P.o_u + (long long)i * nu + k) - al * g;
  }
  for (int k = tw1.lane; k < nx; k += 32) {
    T g = P.nbx ? P.gx[k] * ldc(ec + k) : T(0);
    for (int c = c0; c < c1; ++c) {
      const T* eq = eta + P.e_q + (long long)(c - 1) * P.W;
      if (P.full) {   // (F_Q^c)' eta_Q^c
        const T* F = P.FQ + (size_t)(c - 1) * nx * nx + k;
#pragma unroll 8
        for (int e = 0; e < nx; ++e) g = fma(ldr(F + (size_t)e * nx), ldc(eq + e), g);
      } else {
        g += ldr(P.qh + (long long)(c - 1) * nx + k) * ldc(eq + k);
      }
    }
#pragma unroll 8
    for (int r = 0; r < P.n_g; ++r) g = fma(ldr(P.GgT + (size_t)k * P.n_g + r), ldc(eg + r), g);
    if (P.l1 != T(0)) {   // l1 rows lambda - x, lambda + x (Prop. 2)
      const T* el = eta + P.e_l1 + (long long)i * (1 + 2 * (nx + nu));
      g += ldc(el + 1 + (nx + nu) + k) - ldc(el + 1 + k);
    }
    if (P.soft) g -= ldc(eta + P.e_sf + (long long)i * (3 * (nx + nu) + 2) + 2 * (nx + nu) + 2 + k);
    s_xb[k] = ldc(z + P.o_x + (long long)i * nx + k) - al * g;
  }
  __syncwarp();
  Acc<T, CH> acc;
  acc.zero();
  team_mv<T, CH>(tw1, acc, P.MP + (size_t)i * nu * P.ldP, P.ldP, nu, nx + nu, s_in);
  T* hb = P.hbuf + (long long)i * nx;
  T* eb = P.ebuf + (long long)i * nu;
  const T* kc = P.kc + (long long)i * (nx + nu);
  team_reduce<T, CH>(tw1, acc, nx + nu, s_red, [&](int j, int, T s) {
    if (j < nx) stc(hb + j, (-s - s_xb[j]) + ldr(kc + j));
    else stc(eb + (j - nx), s - ldr(kc + j));
  });
  if (P.tv) s2_block_tv(P, tw1.lane, i, vin, vout, vref, ra);
  else s2_block(P, tw1.lane, i, vin, vout, vref, ra);
  if (P.l1 != T(0)) l1_prep(P, tw1.lane, i, vin, vout, vref, ra);
  if (P.soft) soft_prep(P, tw1.lane, i, vin, vout, vref, ra);
}

template <class T>
__device__ void prep_leaf(const Prob<T>& P, int lane, int j, const T* __restrict__ vin) {
  const int nx = P.nx;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const int jj = j - P.n_nl;
  const T al = P.alpha;
  const T* ecN = eta + P.e_cN + (long long)jj * P.n_cN;
  const T* eqN = eta + P.e_qN + (long long)jj * (nx + 2);
  for (int k = lane; k < nx; k += 32) {
    T g = P.nbx ? P.gN[k] * ldc(ecN + k) : T(0);
    if (P.full) {   // (F_N^j)' eta_QN^j
      const T* F = P.FN + (size_t)jj * nx * nx + k;
#pragma unroll 8
      for (int e = 0; e < nx; ++e) g = fma(ldr(F + (size_t)e * nx), ldc(eqN + e), g);
    } else {
      g += ldr(P.qNh + (long long)jj * nx + k) * ldc(eqN + k);
    }
#pragma unroll 8
    for (int r = 0; r < P.n_gN; ++r) g = fma(ldr(P.GgNT + (size_t)k * P.n_gN + r), ldc(ecN + P.nbx + r), g);
    const T xbar = ldc(z + P.o_x + (long long)j * nx + k) - al * g;
    stc(P.qbuf + (long long)j * nx + k, -xbar);
  }
}

// ---------------------------------------------------------------------------
// Phase B: one segment, bottom-up. The matrix of the next (node, child) pair
// streams into shared memory while the current one is used.
// ---------------------------------------------------------------------------
template <class T, int CH>
__device__ __forceinline__ void mv_any(const Team& tm, Acc<T, CH>& acc, bool smem, const T* M, int ld,
                                       int nrows, int ncols, const T* in) {
  if (smem) team_mv<T, CH, true>(tm, acc, M, ld, nrows, ncols, in);
  else team_mv<T, CH, false>(tm, acc, M, ld, nrows, ncols, in);
}

// ---------------------------------------------------------------------------
// Column-split mat-vec of the sweeps: thread t of a team owns output columns
// j = t + m*nth (m < NP) and runs the whole dot product over the rows, from
// shared memory, with two partial sums to halve the FMA dependency chain. No
// cross-warp reduction is needed.
// ---------------------------------------------------------------------------
constexpr int NPM = 2;   // most output columns per thread in the sweeps

template <class T, int NP>
__device__ __forceinline__ void col_mv_np(const T* __restrict__ M, int ld, int nrows,
                                          const T* __restrict__ in, int t, int nth, int ncols,
                                          T (&acc)[NPM]) {
  T a0[NP], a1[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) { a0[m] = T(0); a1[m] = T(0); }
  // blocks of RB rows: every load of a block is issued before its FMAs, so a
  // matrix read from global memory (too large for the shared-memory pipe) has
  // RB x NP loads in flight per thread instead of two. Even rows go to a0 and
  // odd rows to a1 in order, as in the pairwise loop below.
  constexpr int RB = 16;
  int k = 0;
  for (; k + RB <= nrows; k += RB) {
    T mv[RB][NP], xv[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      xv[r] = in[k + r];
      const T* row = M + (size_t)(k + r) * ld + t;
#pragma unroll
      for (int m = 0; m < NP; ++m) mv[r][m] = (t + m * nth < ncols) ? row[m * nth] : T(0);
    }
#pragma unroll
    for (int r = 0; r < RB; r += 2)
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        if (t + m * nth < ncols) {
          a0[m] = fma(mv[r][m], xv[r], a0[m]);
          a1[m] = fma(mv[r + 1][m], xv[r + 1], a1[m]);
        }
      }
  }
  for (; k + 1 < nrows; k += 2) {
    const T x0 = in[k], x1 = in[k + 1];
    const T* r0 = M + (size_t)k * ld + t;
    const T* r1 = r0 + ld;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      if (t + m * nth < ncols) {
        a0[m] = fma(r0[m * nth], x0, a0[m]);
        a1[m] = fma(r1[m * nth], x1, a1[m]);
      }
    }
  }
  if (k < nrows) {
    const T x0 = in[k];
    const T* r0 = M + (size_t)k * ld + t;
#pragma unroll
    for (int m = 0; m < NP; ++m)
      if (t + m * nth < ncols) a0[m] = fma(r0[m * nth], x0, a0[m]);
  }
#pragma unroll
  for (int m = 0; m < NP; ++m) acc[m] += a0[m] + a1[m];
}

// acc[m] += sum_k M[k*ld + t + m*nth] * in[k]; ceil(ncols / nth) <= NPM (the
// team size is chosen so that 2 * team threads >= nx + nu)
template <class T>
__device__ __forceinline__ void col_mv(const T* M, int ld, int nrows, const T* in, int t, int nth,
                                       int ncols, T (&acc)[NPM]) {
  if (t >= ncols) return;
  if (ncols <= nth) col_mv_np<T, 1>(M, ld, nrows, in, t, nth, ncols, acc);
  else col_mv_np<T, 2>(M, ld, nrows, in, t, nth, ncols, acc);
}

// cycle probe of thread 0 of CTA 0 (sub-phase breakdown of the sweeps); the
// slots live in shared memory and are written to the control block at exit
struct Probe {
  unsigned long long* slots;
  long long t;
  bool on;
  __device__ __forceinline__ void start(unsigned long long* p) {
    on = (blockIdx.x == 0 && threadIdx.x == 0);
    slots = p;
    if (on) t = clock64();
  }
  __device__ __forceinline__ void mark(int k) {
    if (on) {
      const long long n = clock64();
      slots[k] += (unsigned long long)(n - t);
      t = n;
    }
  }
};

// The node list of one segment: lane k of every warp holds node k (top to
// bottom) for k < 32; longer segments read the rest from global memory.
struct SegList {
  int off, len, c0b, c1b, mynode;
  template <class T>
  __device__ __forceinline__ void load(const Prob<T>& P, int s, int lane) {
    const int4 inf = P.seg_info[s];
    off = inf.x; len = inf.y; c0b = inf.z; c1b = inf.w;
    mynode = (lane < len) ? P.seg_nodes[off + lane] : -1;
  }
  template <class T>
  __device__ __forceinline__ int node(const Prob<T>& P, int k) const {
    const int v = __shfl_sync(0xffffffffu, mynode, k & 31);
    return (k < 32) ? v : P.seg_nodes[off + k];
  }
};

// pipeline items: backward = MB of a child; forward = [KT of the node | MF of
// its first child] or MF of a further child (KT part left unused)
template <class T>
__device__ __forceinline__ void issue_B(const Prob<T>& P, const Team& tm, Pipe<T>& pp, int b, int c) {
  const size_t st = (size_t)P.nx * P.ldB;
  pp.issue(tm, b, P.MB + (size_t)(c - 1) * st, (unsigned)(st * sizeof(T)));
}
template <class T>
__device__ __forceinline__ void issue_F(const Prob<T>& P, const Team& tm, Pipe<T>& pp, int b, int node,
                                        int c, bool with_kt) {
  const size_t ks = (size_t)P.nx * P.ldK, fs = (size_t)(P.nx + P.nu) * P.ldF;
  if (tm.tid == 0) {
    fence_proxy_async();
    mbar_expect_tx(pp.bar + b, (unsigned)(((with_kt ? ks : 0) + fs) * sizeof(T)));
    if (with_kt) bulk_g2s(pp.buf[b], P.KT + (size_t)node * ks, (unsigned)(ks * sizeof(T)), pp.bar + b);
    bulk_g2s(pp.buf[b] + ks, P.MF + (size_t)(c - 1) * fs, (unsigned)(fs * sizeof(T)), pp.bar + b);
  }
}
template <class T, int CH>
__device__ __forceinline__ void issue_first_B(const Prob<T>& P, const Team& tm, Pipe<T>& pp, int s) {
  issue_B(P, tm, pp, pp.cur, P.seg_info[s].z);
}
template <class T, int CH>
__device__ __forceinline__ void issue_first_F(const Prob<T>& P, const Team& tm, Pipe<T>& pp, int s) {
  const int top = P.seg_top[s];
  const int4 inf = P.seg_info[s];
  const int c0 = (inf.y > 1) ? P.seg_nodes[inf.x + 1] : inf.z;
  issue_F(P, tm, pp, pp.cur, top, c0, true);
}

// ---------------------------------------------------------------------------
// Phase B: one segment, bottom-up. s_a, s_b: ping-pong carry buffers (D each).
// ---------------------------------------------------------------------------
template <class T, int CH>
__device__ bool backward_segment(const Prob<T>& P, const Team& tm, T* s_a, T* s_b, Pipe<T>& pp,
                                 int* err, int s, bool prefetched, unsigned long long* prof) {
  Probe pr;
  pr.start(prof);
  const int nx = P.nx, nu = P.nu, w = nx + nu, ldB = P.ldB;
  const int t = tm.tid, nth = tm.nth;
  const size_t mstride = (size_t)nx * ldB;
  const T* __restrict__ MB = P.MB;
  T* __restrict__ qbuf = P.qbuf;
  T* __restrict__ dbuf = P.dbuf;
  const T* __restrict__ hbuf = P.hbuf;
  const T* __restrict__ ebuf = P.ebuf;
  bool ok = true;
  if (pp.on && !prefetched) issue_first_B<T, CH>(P, tm, pp, s);
  SegList sl;
  sl.load(P, s, tm.lane);
  const int len = sl.len;
  auto load_pre = [&](int node, T (&dst)[NPM]) {
#pragma unroll
    for (int m = 0; m < NPM; ++m) {
      const int j = t + m * nth;
      dst[m] = (j < nx) ? ldc(hbuf + (long long)node * nx + j)
                        : ((j < w) ? ldc(ebuf + (long long)node * nu + (j - nx)) : T(0));
    }
  };
  int i = sl.node(P, len - 1);
  T pre[NPM];
  load_pre(i, pre);
  T* cin = s_a;    // carry read by this step
  T* cout = s_b;   // carry written by this step
  for (int step = 0; step < len; ++step) {
    const bool bottom = (step == 0);
    const int c0 = bottom ? sl.c0b : sl.node(P, len - step);
    const int c1 = bottom ? sl.c1b : c0 + 1;
    const int inext = (step + 1 < len) ? sl.node(P, len - 2 - step) : -1;
    T pren[NPM];
    if (inext >= 0) load_pre(inext, pren);
    T acc[NPM];
#pragma unroll
    for (int m = 0; m < NPM; ++m) acc[m] = T(0);
    for (int c = c0; c < c1; ++c) {
      if (bottom) {   // q of the child from global memory (computed by another team or a leaf)
        for (int k = t; k < nx; k += nth) cin[k] = ldc(qbuf + (long long)c * nx + k);
      }
      pr.mark(11);
      if (pp.on) {
        if (!pp.wait(tm, pp.cur, err, pp.okp, pp.diag, 1)) return false;   // includes a team barrier
      } else {
        tm.sync();
      }
      pr.mark(8);
      // next item into the other buffer (read before the barrier just passed)
      const int cn = (c + 1 < c1) ? c + 1 : ((inext >= 0) ? i : -1);
      if (pp.on && cn > 0) issue_B(P, tm, pp, pp.cur ^ 1, cn);
      const T* Mb = pp.on ? pp.buf[pp.cur] : MB + (size_t)(c - 1) * mstride;
      col_mv<T>(Mb, ldB, nx, cin, t, nth, w, acc);
      if (pp.on) pp.cur ^= 1;
      pr.mark(9);
      if (bottom && c + 1 < c1) tm.sync();       // cin is reloaded for the next child
    }
#pragma unroll
    for (int m = 0; m < NPM; ++m) {
      const int j = t + m * nth;
      if (j < nx) {
        const T qq = acc[m] + pre[m];
        cout[j] = qq;
        stc(qbuf + (long long)i * nx + j, qq);
      } else if (j < w) {
        stc(dbuf + (long long)i * nu + (j - nx), pre[m] - acc[m]);
      }
    }
    tm.sync();
    pr.mark(10);
    T* tt = cin; cin = cout; cout = tt;
    if (inext >= 0) {
#pragma unroll
      for (int m = 0; m < NPM; ++m) pre[m] = pren[m];
    }
    i = inext;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Phase F: one segment, top-down (x and u of z+ only; their residuals and the
// eta update follow in phase E). The team's input buffer holds [x^i ; d^i].
// Threads [0, nx) compute x of the child, threads [nx, nx + nu) compute u^i
// when the team is wide enough; otherwise every thread does both in turn.
// ---------------------------------------------------------------------------
template <class T, int CH>
__device__ bool forward_segment(const Prob<T>& P, const Team& tm, T* s_a, T* s_b, Pipe<T>& pp,
                                int* err, int s, T* __restrict__ vout, bool prefetched) {
  const int nx = P.nx, nu = P.nu, w = nx + nu, ldF = P.ldF, ldK = P.ldK;
  const int t = tm.tid, nth = tm.nth;
  const size_t ks = (size_t)nx * ldK;
  const T* __restrict__ dbuf = P.dbuf;
  const T* __restrict__ cvec = P.cvec;
  const long long o_x = P.o_x, o_u = P.o_u;
  const bool wide = nth >= w;
  const size_t fs = (size_t)w * ldF;
  bool ok = true;
  if (pp.on && !prefetched) issue_first_F<T, CH>(P, tm, pp, s);
  SegList sl;
  sl.load(P, s, tm.lane);
  const int len = sl.len;
  auto first_child = [&](int k) { return (k + 1 < len) ? sl.node(P, k + 1) : sl.c0b; };
  int i = sl.node(P, 0);
  T* cin = s_a;
  T* cout = s_b;
  // input of the first step: x^i (fixed x0 at the root) and d^i
  for (int k = t; k < w; k += nth) {
    T v;
    if (k < nx) {
      if (i == 0) {
        v = P.x0s[k];
        stc(vout + o_x + k, zc_add(P, o_x + k, v));
      } else {
        const long long ix = o_x + (long long)i * nx + k;
        v = zc_sub(P, ix, ldc(vout + ix));
      }
    } else {
      v = ldc(dbuf + (long long)i * nu + (k - nx));
    }
    cin[k] = v;
  }
  T cp[NPM];
  {
    const int c = first_child(0);
#pragma unroll
    for (int m = 0; m < NPM; ++m) {
      const int j = t + m * nth;
      cp[m] = (j < nx) ? ldr(cvec + (long long)(c - 1) * nx + j) : T(0);
    }
  }
  for (int step = 0; step < len; ++step) {
    const bool chain = (step + 1 < len);
    const int c0 = first_child(step);
    const int c1 = chain ? c0 + 1 : sl.c1b;
    // prefetch d of the next node and c of its first child
    T dpn[NPM], cpn[NPM];
    if (chain) {
      const int cn = first_child(step + 1);
#pragma unroll
      for (int m = 0; m < NPM; ++m) {
        const int j = t + m * nth;
        dpn[m] = (j < nu) ? ldc(dbuf + (long long)c0 * nu + j) : T(0);
        cpn[m] = (j < nx) ? ldr(cvec + (long long)(cn - 1) * nx + j) : T(0);
      }
    }
    for (int c = c0; c < c1; ++c) {
      if (pp.on) {
        if (!pp.wait(tm, pp.cur, err, pp.okp, pp.diag, 2)) return false;      // includes a team barrier
        if (c + 1 < c1) issue_F(P, tm, pp, pp.cur ^ 1, i, c + 1, false);
        else if (chain) issue_F(P, tm, pp, pp.cur ^ 1, c0, first_child(step + 1), true);
      } else {
        tm.sync();
      }
      const T* KTb = pp.on ? pp.buf[pp.cur] : P.KT + (size_t)i * ks;
      const T* MFb = pp.on ? KTb + ks : P.MF + (size_t)(c - 1) * fs;
      if (c > c0) {
#pragma unroll
        for (int m = 0; m < NPM; ++m) {
          const int j = t + m * nth;
          cp[m] = (j < nx) ? ldr(cvec + (long long)(c - 1) * nx + j) : T(0);
        }
      }
      // x^c = Abar_c x^i + B_c d^i + c_c
      T ax[NPM];
#pragma unroll
      for (int m = 0; m < NPM; ++m) ax[m] = T(0);
      if (wide) {
        if (t < nx) col_mv<T>(MFb, ldF, w, cin, t, nth, nx, ax);
      } else {
        col_mv<T>(MFb, ldF, w, cin, t, nth, nx, ax);
      }
#pragma unroll
      for (int m = 0; m < NPM; ++m) {
        const int j = t + m * nth;
        if (j < nx) {
          const T xc = ax[m] + cp[m];
          const long long ix = o_x + (long long)c * nx + j;
          stc(vout + ix, zc_add(P, ix, xc));
          if (chain) cout[j] = xc;
        }
      }
      // u^i = K x^i + d^i, once per node
      if (c == c0) {
        T au[NPM];
#pragma unroll
        for (int m = 0; m < NPM; ++m) au[m] = T(0);
        if (wide) {
          if (t >= nx && t < w) {
            const int tu = t - nx;
            col_mv<T>(KTb, ldK, nx, cin, tu, nth, nu, au);
            const long long iu = o_u + (long long)i * nu + tu;
            stc(vout + iu, zc_add(P, iu, au[0] + cin[nx + tu]));
          }
        } else {
          col_mv<T>(KTb, ldK, nx, cin, t, nth, nu, au);
#pragma unroll
          for (int m = 0; m < NPM; ++m) {
            const int j = t + m * nth;
            if (j < nu) {
              const long long iu = o_u + (long long)i * nu + j;
              stc(vout + iu, zc_add(P, iu, au[m] + cin[nx + j]));
            }
          }
        }
      }
      if (pp.on) pp.cur ^= 1;
    }
    if (chain) {
#pragma unroll
      for (int m = 0; m < NPM; ++m) {
        const int j = t + m * nth;
        if (j < nu) cout[nx + j] = dpn[m];
        cp[m] = cpn[m];
      }
      tm.sync();
      T* tt = cin; cin = cout; cout = tt;
      i = c0;
    }
  }
  tm.sync();   // the input buffers are reused by the team's next segment
  return ok;
}

// z residual of the x (and u) of one node, accumulated by one warp (phase E)
template <class T>
__device__ __forceinline__ void z_resid(const T* __restrict__ vin, const T* __restrict__ vout,
                                        const T* __restrict__ vref, long long off, int len,
                                        int lane, RedAcc<T>& ra) {
  for (int k = lane; k < len; k += 32) {
    const T o = ldc(vin + off + k);
    ra.z(o, ldc(vout + off + k), dirv(vref, off + k));
  }
}

// ---------------------------------------------------------------------------
// Phase E: eta blocks (one warp each); x, u, y, tau, s of z+ are read from vout
// ---------------------------------------------------------------------------
// prox step of one element ie of eta whose set C is a product of intervals:
// eta+ = eb - alpha proj_C(eb / alpha). In the centred form eb is the
// increment over the centre, the argument and the step are formed in FP64
// about the centre, and the increment eta+ - eta_c is returned.
template <class T, class PF>
__device__ __forceinline__ T eta_prox(const Prob<T>& P, long long ie, T eb, PF&& proj) {
  if (P.ctrA) {
    const double w = fma((double)eb, P.ctr_ial, ldr(P.ctrA + ie));
    return (T)fma(-P.ctr_al, proj(w), ldr(P.ctrB + ie) + (double)eb);
  }
  const T al = P.alpha;
  const T w = eb / al;
  return eb - al * proj(w);
}

template <class T>
__device__ void eta_nonleaf(const Prob<T>& P, int lane, int i, const T* __restrict__ vin,
                            T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  T* eo = vout + P.nz;
  const T* er = vref ? vref + P.nz : nullptr;
  const int c0 = P.ch_off[i], m = P.ch_off[i + 1] - c0;
  const T al = P.alpha;
  const long long yo = P.o_y + P.yoff[i];
  const long long ye = P.e_y + P.yoff[i];
  // y part: (K^i)* = R^{npos}_+ x R (AV@R: npos = 2m; total variation: 3m + 1)
  const int ly = (int)(P.yoff[i + 1] - P.yoff[i]), npos = risk_npos(P, m);
  for (int e = lane; e < ly; e += 32) {
    const T Lo = ldc(z + yo + e), Ln = ldc(vout + yo + e);
    const T eo_ = ldc(eta + ye + e);
    const T eb = eo_ + al * (T(2) * Ln - Lo);
    const bool cone = e < npos;
    const T en = eta_prox(P, ye + e, eb, [&](auto w) { return cone ? max(w, decltype(w)(0)) : w; });
    stc(eo + ye + e, en);
    ra.eta(eo_, en, er ? ldc(er + ye + e) : T(0), Lo - Ln, dirv(vref, yo + e));
  }
  // s part: s^i - b'y^i in R_+
  {
    T bo = 0, bn = 0, bd = 0, brd = 0;   // b'y of old and new, b'(y_old - y_new), b'(direction y)
    for (int k = lane; k < ly; k += 32) {
      const T p = risk_b(P, i, c0, m, k);
      const T o = ldc(z + yo + k), nn = ldc(vout + yo + k);
      bo += p * o;
      bn += p * nn;
      bd += p * (o - nn);
      brd += p * dirv(vref, yo + k);
    }
    bo = warp_sum(bo); bn = warp_sum(bn); bd = warp_sum(bd); brd = warp_sum(brd);
    if (lane == 0) {
      const long long is = (i == 0) ? 0 : P.o_s + i - 1;
      const T so = ldc(z + is);
      const T sn = ldc(vout + is);
      const T Lo = so - bo;
      const T Ln = sn - bn;
      const T lrz = (so - sn) - bd;
      const T lod = vref ? ldc(vref + is) - brd : T(0);
      const long long ie = P.e_s + i;
      const T eo_ = ldc(eta + ie);
      const T eb = eo_ + al * (T(2) * Ln - Lo);
      const T en = eta_prox(P, ie, eb, [&](auto w) { return max(w, decltype(w)(0)); });
      stc(eo + ie, en);
      ra.eta(eo_, en, er ? ldc(er + ie) : T(0), lrz, lod);
    }
  }
  if (P.n_c == 0) return;
  const long long ce = P.e_c + (long long)i * P.n_c;
  const long long xo = P.o_x + (long long)i * nx;
  const long long uo = P.o_u + (long long)i * nu;
  // box rows
  for (int e = lane; e < P.nbox; e += 32) {
    T g;
    long long idx;
    if (e < P.nbx) {
      g = P.gx[e]; idx = xo + e;
    } else {
      g = P.gu[e - P.nbx]; idx = uo + (e - P.nbx);
    }
    const T o = ldc(z + idx), nn = ldc(vout + idx);
    const T Lo = g * o, Ln = g * nn;
    const T eo_ = ldc(eta + ce + e);
    const T eb = eo_ + al * (T(2) * Ln - Lo);
    const T lo = P.box_lo[(long long)i * P.nbox + e], hi = P.box_hi[(long long)i * P.nbox + e];
    const T en = eta_prox(P, ce + e, eb, [&](auto w) {
      using V = decltype(w);
      return min(max(w, (V)lo), (V)hi);
    });
    stc(eo + ce + e, en);
    ra.eta(eo_, en, er ? ldc(er + ce + e) : T(0), g * (o - nn), g * dirv(vref, idx));
  }
  // ball rows on u
  if (P.has_ball) {
    const bool ctr = P.ctrA != nullptr;
    double n2 = 0;   // FP64 in the centred form, where w is formed about the centre
    for (int k = lane; k < nu; k += 32) {
      const T g = P.gu[k];
      const long long ie = ce + P.nbox + k;
      const T eb = ldc(eta + ie) + al * (T(2) * g * ldc(vout + uo + k) - g * ldc(z + uo + k));
      if (ctr) {
        const double w = fma((double)eb, P.ctr_ial, ldr(P.ctrA + ie));
        n2 = fma(w, w, n2);
      } else {
        const T w = eb / al;
        n2 = (double)((T)n2 + w * w);
      }
    }
    const double r = (double)P.ball[i];
    double sc = 1.0;
    T scT = T(1);
    if (ctr) {
      const double nw = sqrt(warp_sum(n2));
      sc = (nw > r) ? r / nw : 1.0;
    } else {
      const T nw = sqrt(warp_sum((T)n2));
      scT = (nw > (T)r) ? (T)r / nw : T(1);
    }
    for (int k = lane; k < nu; k += 32) {
      const T g = P.gu[k];
      const T o = ldc(z + uo + k), nn = ldc(vout + uo + k);
      const T Lo = g * o, Ln = g * nn;
      const long long ie = ce + P.nbox + k;
      const T eo_ = ldc(eta + ie);
      const T eb = eo_ + al * (T(2) * Ln - Lo);
      const T en = ctr ? eta_prox(P, ie, eb, [&](auto w) { return w * (decltype(w))sc; })
                       : eta_prox(P, ie, eb, [&](auto w) { return w * (decltype(w))scT; });
      stc(eo + ie, en);
      ra.eta(eo_, en, er ? ldc(er + ie) : T(0), g * (o - nn), g * dirv(vref, uo + k));
    }
  }
  // general rows Gx x^i + Gu u^i in a box
  if (P.n_g) {
    const long long ge = ce + P.nbox + (P.has_ball ? nu : 0);
    for (int r = lane; r < P.n_g; r += 32) {
      const T* G = P.Gg + (size_t)r * (nx + nu);
      T Lo = 0, Ln = 0, Ld = 0, Lrd = 0;
#pragma unroll 8
      for (int k = 0; k < nx + nu; ++k) {
        const long long idx = (k < nx) ? xo + k : uo + (k - nx);
        const T g = ldr(G + k);
        const T o = ldc(z + idx), nn = ldc(vout + idx);
        Lo = fma(g, o, Lo);
        Ln = fma(g, nn, Ln);
        Ld = fma(g, o - nn, Ld);
        Lrd = fma(g, dirv(vref, idx), Lrd);
      }
      const T eo_ = ldc(eta + ge + r);
      const T eb = eo_ + al * (T(2) * Ln - Lo);
      const T lo = P.gen_lo[(long long)i * P.n_g + r], hi = P.gen_hi[(long long)i * P.n_g + r];
      const T en = eta_prox(P, ge + r, eb, [&](auto w) {
        using V = decltype(w);
        return min(max(w, (V)lo), (V)hi);
      });
      stc(eo + ge + r, en);
      ra.eta(eo_, en, er ? ldc(er + ge + r) : T(0), Ld, Lrd);
    }
  }
}

// The l1 rows of non-leaf node i (Prop. 2): theta - sum_k w_k lambda_k,
// lambda - z, lambda + z (z = (x^i, u^i)), each in R_+.
template <class T>
__device__ void eta_l1(const Prob<T>& P, int lane, int i, const T* __restrict__ vin, T* __restrict__ vout,
                       const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu, d = nx + nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  T* eo = vout + P.nz;
  const T* er = vref ? vref + P.nz : nullptr;
  const T al = P.alpha;
  const long long le = P.e_l1 + (long long)i * (1 + 2 * d);
  const long long ol = P.o_lam + (long long)i * d;
  auto pos = [](auto w) { return max(w, decltype(w)(0)); };
  auto row = [&](long long ie, T Lo, T Ln, T Ld, T Lrd) {
    const T eo_ = ldc(eta + ie);
    const T eb = eo_ + al * (T(2) * Ln - Lo);
    const T en = eta_prox(P, ie, eb, pos);
    stc(eo + ie, en);
    ra.eta(eo_, en, er ? ldc(er + ie) : T(0), Ld, Lrd);
  };
  T so = 0, sn = 0, sd = 0, sr = 0;
  for (int k = lane; k < d; k += 32) {
    const T w = ldr(P.l1w + k);
    const T lo = ldc(z + ol + k), ln = ldc(vout + ol + k), lr = dirv(vref, ol + k);
    so += w * lo; sn += w * ln; sd += w * (lo - ln); sr += w * lr;
    const long long iz = (k < nx) ? P.o_x + (long long)i * nx + k : P.o_u + (long long)i * nu + (k - nx);
    const T zo = ldc(z + iz), zn = ldc(vout + iz), zr = dirv(vref, iz);
    row(le + 1 + k, lo - zo, ln - zn, (lo - ln) - (zo - zn), lr - zr);
    row(le + 1 + d + k, lo + zo, ln + zn, (lo - ln) + (zo - zn), lr + zr);
  }
  so = warp_sum(so); sn = warp_sum(sn); sd = warp_sum(sd); sr = warp_sum(sr);
  if (lane == 0) {
    const long long ith = P.o_th + i;
    const T tho = ldc(z + ith), thn = ldc(vout + ith), thr = dirv(vref, ith);
    row(le, tho - so, thn - sn, (tho - thn) - sd, thr - sr);
  }
}

// Cost cone block in the centred form: ebv holds the increments of
// eta_bar = eta + alpha L(2 z+ - z) over the centre; w = eta_bar/alpha - a is
// formed in FP64 about the centre (ctrA folds in -a), projected on the
// second-order cone in FP64, and the increment of eta+ = eta_bar - alpha (a +
// Pi(w)) over eta_c is stored (ctrB folds in -alpha a).
template <class T, int NE>
__device__ __forceinline__ void soc_centred(const Prob<T>& P, int lane, int dim, long long ebase,
                                            const T* __restrict__ eta, T* __restrict__ eo,
                                            const T* __restrict__ er, const T (&ebv)[NE], const T (&ldv)[NE],
                                            const T (&lrv)[NE], RedAcc<T>& ra) {
  double wv[NE];
  double n2 = 0.0, tt = 0.0;
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    wv[q] = 0.0;
    if (e < dim) {
      wv[q] = fma((double)ebv[q], P.ctr_ial, ldr(P.ctrA + ebase + e));
      if (e < dim - 1) n2 = fma(wv[q], wv[q], n2);
      else tt = wv[q];
    }
  }
  const double nw = sqrt(warp_sum(n2));
  const double t = __shfl_sync(0xffffffffu, tt, (dim - 1) & 31);
  const int cs = (nw <= t) ? 0 : ((nw <= -t) ? 1 : 2);
  const double f = 0.5 * (nw + t);
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    if (e < dim) {
      double ps;
      if (cs == 0) ps = wv[q];
      else if (cs == 1) ps = 0.0;
      else ps = (e < dim - 1) ? wv[q] * (f / nw) : f;
      const T en = (T)fma(-P.ctr_al, ps, ldr(P.ctrB + ebase + e) + (double)ebv[q]);
      const T eo_ = ldc(eta + ebase + e);
      stc(eo + ebase + e, en);
      ra.eta(eo_, en, er ? ldc(er + ebase + e) : T(0), ldv[q], lrv[q]);
    }
  }
}

// translated SOC cost block: a + Pi_SOC(eb/alpha - a), a = (0.., 1/2, -1/2)
// acst: the block's translation a (null: (0, .., 1/2, -1/2))
template <class T>
__device__ __forceinline__ T soc_a(const T* acst, int e, int dim) {
  if (acst) return ldr(acst + e);
  return (e == dim - 2) ? T(0.5) : ((e == dim - 1) ? T(-0.5) : T(0));
}

template <class T, int NE, class FL>
__device__ __forceinline__ void soc_block(const Prob<T>& P, int lane, int dim, long long ebase,
                                          const T* __restrict__ eta, T* __restrict__ eo,
                                          const T* __restrict__ er, FL&& Lz, RedAcc<T>& ra,
                                          const T* acst = nullptr) {
  const T al = P.alpha;
  T ebv[NE];
  T n2 = 0, tt = 0;
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    ebv[q] = 0;
    if (e < dim) {
      T Lo, Ln, Ld, Lrd;
      Lz(e, Lo, Ln, Ld, Lrd);
      const T eb = ldc(eta + ebase + e) + al * (T(2) * Ln - Lo);
      ebv[q] = eb;
      const T ae = soc_a(acst, e, dim);
      const T w = eb / al - ae;
      if (e < dim - 1) n2 += w * w;
      else tt = w;
    }
  }
  if (P.ctrA) {   // centred form: the projection about the centre in FP64
    T ldv[NE], lrv[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int e = lane + 32 * q;
      ldv[q] = T(0);
      lrv[q] = T(0);
      if (e < dim) {
        T Lo, Ln;
        Lz(e, Lo, Ln, ldv[q], lrv[q]);
      }
    }
    soc_centred<T, NE>(P, lane, dim, ebase, eta, eo, er, ebv, ldv, lrv, ra);
    return;
  }
  const T nw = sqrt(warp_sum(n2));
  const T t = __shfl_sync(0xffffffffu, tt, (dim - 1) & 31);
  // case 0: inside (keep), 1: polar (zero), 2: boundary
  const int cs = (nw <= t) ? 0 : ((nw <= -t) ? 1 : 2);
  const T f = (nw + t) / T(2);
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    if (e < dim) {
      T Lo, Ln, Ld, Lrd;
      Lz(e, Lo, Ln, Ld, Lrd);
      const T eb = ebv[q];
      const T ae = soc_a(acst, e, dim);
      const T w = eb / al - ae;
      T ps;
      if (cs == 0) ps = w;
      else if (cs == 1) ps = T(0);
      else ps = (e < dim - 1) ? w * (f / nw) : f;
      const T en = eb - al * (ae + ps);
      const T eo_ = ldc(eta + ebase + e);
      stc(eo + ebase + e, en);
      ra.eta(eo_, en, er ? ldc(er + ebase + e) : T(0), Ld, Lrd);
    }
  }
}

// Translated cost cone of a block with full factors: the caller has the
// block's eta_bar = eta + alpha L(2 z+ - z) (ebv), L(z - z+) (ldv) and
// L(direction) (lrv) per lane element e = lane + 32 q.
template <class T, int NE>
__device__ __forceinline__ void soc_block_vals(const Prob<T>& P, int lane, int dim, long long ebase,
                                               const T* __restrict__ eta, T* __restrict__ eo,
                                               const T* __restrict__ er, const T (&ebv)[NE], const T (&ldv)[NE],
                                               const T (&lrv)[NE], const T* acst, RedAcc<T>& ra) {
  if (P.ctrA) {
    soc_centred<T, NE>(P, lane, dim, ebase, eta, eo, er, ebv, ldv, lrv, ra);
    return;
  }
  const T al = P.alpha;
  T n2 = 0, tt = 0;
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    if (e < dim) {
      const T w = ebv[q] / al - soc_a(acst, e, dim);
      if (e < dim - 1) n2 += w * w;
      else tt = w;
    }
  }
  const T nw = sqrt(warp_sum(n2));
  const T t = __shfl_sync(0xffffffffu, tt, (dim - 1) & 31);
  const int cs = (nw <= t) ? 0 : ((nw <= -t) ? 1 : 2);
  const T f = (nw + t) / T(2);
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    if (e < dim) {
      const T ae = soc_a(acst, e, dim);
      const T w = ebv[q] / al - ae;
      T ps;
      if (cs == 0) ps = w;
      else if (cs == 1) ps = T(0);
      else ps = (e < dim - 1) ? w * (f / nw) : f;
      const T en = ebv[q] - al * (ae + ps);
      const T eo_ = ldc(eta + ebase + e);
      stc(eo + ebase + e, en);
      ra.eta(eo_, en, er ? ldc(er + ebase + e) : T(0), ldv[q], lrv[q]);
    }
  }
}

// per lane element e = lane + 32 q < m: acc1 += F (2 z_new - z_old),
// acc2 += F (z_old - z_new), acc3 += F dir, for F given by its transpose FT
// (m x m row-major: FT[k m + e] = F[e][k]) acting on z at offset zo; elements
// are placed at e + shift of the arrays
template <class T, int NE>
__device__ __forceinline__ void full_mv3(int lane, int m, int shift, const T* __restrict__ FT, const T* __restrict__ z,
                                         const T* __restrict__ vout, const T* __restrict__ vref, long long zo,
                                         T (&a1)[NE], T (&a2)[NE], T (&a3)[NE]) {
  for (int k = 0; k < m; ++k) {
    const T o = ldc(z + zo + k), nn = ldc(vout + zo + k);
    const T x1 = T(2) * nn - o, x2 = o - nn, x3 = dirv(vref, zo + k);
    const T* Fk = FT + (size_t)k * m;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int e = lane + 32 * q - shift;
      if (e >= 0 && e < m) {
        const T f = ldr(Fk + e);
        a1[q] = fma(f, x1, a1[q]);
        a2[q] = fma(f, x2, a2[q]);
        a3[q] = fma(f, x3, a3[q]);
      }
    }
  }
}

template <class T, int NE>
__device__ void eta_soc_full(const Prob<T>& P, int lane, int c, const T* __restrict__ vin,
                             T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu, W = P.W;
  const int i = P.anc[c];
  const T* z = vin;
  const T* eta = vin + P.nz;
  const long long ebase = P.e_q + (long long)(c - 1) * W;
  T a1[NE], a2[NE], a3[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) { a1[q] = T(0); a2[q] = T(0); a3[q] = T(0); }
  full_mv3<T, NE>(lane, nx, 0, P.FQT + (size_t)(c - 1) * nx * nx, z, vout, vref, P.o_x + (long long)i * nx, a1, a2, a3);
  full_mv3<T, NE>(lane, nu, nx, P.FRT + (size_t)(c - 1) * nu * nu, z, vout, vref, P.o_u + (long long)i * nu, a1, a2,
                  a3);
  const long long it = P.o_tau + c - 1;
  T to = ldc(z + it), tn = ldc(vout + it), td = dirv(vref, it);
  if (P.l1 != T(0)) {   // (tau^c - lambda_0 theta^i)/2 (Prop. 2)
    const long long ith = P.o_th + i;
    to -= P.l1 * ldc(z + ith); tn -= P.l1 * ldc(vout + ith); td -= P.l1 * dirv(vref, ith);
  }
  if (P.soft) {   // (tau^c - sigma^i)/2
    const long long isg = P.o_sg + i;
    to -= ldc(z + isg); tn -= ldc(vout + isg); td -= dirv(vref, isg);
  }
  const T al = P.alpha;
  T ebv[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    if (e >= nx + nu && e < W) {   // tau/2 twice
      a1[q] = T(0.5) * (T(2) * tn - to);
      a2[q] = T(0.5) * (to - tn);
      a3[q] = T(0.5) * td;
    }
    ebv[q] = (e < W) ? ldc(eta + ebase + e) + al * a1[q] : T(0);
  }
  soc_block_vals<T, NE>(P, lane, W, ebase, eta, vout + P.nz, vref ? vref + P.nz : nullptr, ebv, a2, a3,
                        P.acost ? P.acost + (size_t)(c - 1) * W : nullptr, ra);
}

template <class T, int NE>
__device__ void eta_leaf_full_cone(const Prob<T>& P, int lane, int j, const T* __restrict__ vin,
                                   T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, dim = nx + 2;
  const int jj = j - P.n_nl;
  const T* z = vin;
  const T* eta = vin + P.nz;
  const long long ebase = P.e_qN + (long long)jj * dim;
  T a1[NE], a2[NE], a3[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) { a1[q] = T(0); a2[q] = T(0); a3[q] = T(0); }
  full_mv3<T, NE>(lane, nx, 0, P.FNT + (size_t)jj * nx * nx, z, vout, vref, P.o_x + (long long)j * nx, a1, a2, a3);
  const long long is = P.o_s + j - 1;
  const T so = ldc(z + is), sn = ldc(vout + is), sd = dirv(vref, is);
  const T al = P.alpha;
  T ebv[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    if (e >= nx && e < dim) {   // s/2 twice
      a1[q] = T(0.5) * (T(2) * sn - so);
      a2[q] = T(0.5) * (so - sn);
      a3[q] = T(0.5) * sd;
    }
    ebv[q] = (e < dim) ? ldc(eta + ebase + e) + al * a1[q] : T(0);
  }
  soc_block_vals<T, NE>(P, lane, dim, ebase, eta, vout + P.nz, vref ? vref + P.nz : nullptr, ebv, a2, a3,
                        P.acostN ? P.acostN + (size_t)jj * dim : nullptr, ra);
}

template <class T, int NE>
__device__ void eta_soc(const Prob<T>& P, int lane, int c, const T* __restrict__ vin,
                        T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu;
  const int i = P.anc[c];
  const T* z = vin;
  const long long xo = P.o_x + (long long)i * nx, uo = P.o_u + (long long)i * nu;
  const long long it = P.o_tau + c - 1;
  const T* qh = P.qh + (long long)(c - 1) * nx;
  const T* rh = P.rh + (long long)(c - 1) * nu;
  // with an l1 term the last two entries are (tau^c - lambda_0 theta^i)/2 (Prop. 2)
  T tho = 0, thn = 0, thd = 0;
  if (P.l1 != T(0)) {
    const long long ith = P.o_th + i;
    tho = P.l1 * ldc(z + ith); thn = P.l1 * ldc(vout + ith); thd = P.l1 * dirv(vref, ith);
  }
  if (P.soft) {   // (tau^c - sigma^i)/2
    const long long isg = P.o_sg + i;
    tho += ldc(z + isg); thn += ldc(vout + isg); thd += dirv(vref, isg);
  }
  auto Lz = [&](int e, T& Lo, T& Ln, T& Ld, T& Lrd) {
    long long idx;
    T g;
    if (e < nx) {
      g = ldr(qh + e); idx = xo + e;
    } else if (e < nx + nu) {
      g = ldr(rh + (e - nx)); idx = uo + (e - nx);
    } else {
      g = T(0.5); idx = it;
    }
    T o = ldc(z + idx), nn = ldc(vout + idx), dd = dirv(vref, idx);
    if (e >= nx + nu) { o -= tho; nn -= thn; dd -= thd; }
    Lo = g * o; Ln = g * nn; Ld = g * (o - nn); Lrd = g * dd;
  };
  soc_block<T, NE>(P, lane, P.W, P.e_q + (long long)(c - 1) * P.W, vin + P.nz, vout + P.nz,
                   vref ? vref + P.nz : nullptr, Lz, ra, P.acost ? P.acost + (size_t)(c - 1) * P.W : nullptr);
}

template <class T, int NE>
__device__ void eta_leaf(const Prob<T>& P, int lane, int j, const T* __restrict__ vin,
                         T* __restrict__ vout, const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx;
  const T* z = vin;
  const T* eta = vin + P.nz;
  T* eo = vout + P.nz;
  const T* er = vref ? vref + P.nz : nullptr;
  const int jj = j - P.n_nl;
  const long long xo = P.o_x + (long long)j * nx;
  const T al = P.alpha;
  if (P.nbx) {
    const long long ce = P.e_cN + (long long)jj * P.n_cN;
    for (int e = lane; e < nx; e += 32) {
      const T g = P.gN[e], o = ldc(z + xo + e), nn = ldc(vout + xo + e);
      const T Lo = g * o, Ln = g * nn;
      const T eo_ = ldc(eta + ce + e);
      const T eb = eo_ + al * (T(2) * Ln - Lo);
      const T lo = P.boxN_lo[(long long)jj * nx + e], hi = P.boxN_hi[(long long)jj * nx + e];
      const T en = eta_prox(P, ce + e, eb, [&](auto w) {
        using V = decltype(w);
        return min(max(w, (V)lo), (V)hi);
      });
      stc(eo + ce + e, en);
      ra.eta(eo_, en, er ? ldc(er + ce + e) : T(0), g * (o - nn), g * dirv(vref, xo + e));
    }
  }
  // general rows GN x^j in a box
  if (P.n_gN) {
    const long long ge = P.e_cN + (long long)jj * P.n_cN + P.nbx;
    for (int r = lane; r < P.n_gN; r += 32) {
      const T* G = P.GgN + (size_t)r * nx;
      T Lo = 0, Ln = 0, Ld = 0, Lrd = 0;
#pragma unroll 8
      for (int k = 0; k < nx; ++k) {
        const T g = ldr(G + k);
        const T o = ldc(z + xo + k), nn = ldc(vout + xo + k);
        Lo = fma(g, o, Lo);
        Ln = fma(g, nn, Ln);
        Ld = fma(g, o - nn, Ld);
        Lrd = fma(g, dirv(vref, xo + k), Lrd);
      }
      const T eo_ = ldc(eta + ge + r);
      const T eb = eo_ + al * (T(2) * Ln - Lo);
      const T lo = P.genN_lo[(long long)jj * P.n_gN + r], hi = P.genN_hi[(long long)jj * P.n_gN + r];
      const T en = eta_prox(P, ge + r, eb, [&](auto w) {
        using V = decltype(w);
        return min(max(w, (V)lo), (V)hi);
      });
      stc(eo + ge + r, en);
      ra.eta(eo_, en, er ? ldc(er + ge + r) : T(0), Ld, Lrd);
    }
  }
  if (P.full) {
    eta_leaf_full_cone<T, NE>(P, lane, j, vin, vout, vref, ra);
    return;
  }
  const long long is = P.o_s + j - 1;
  const T* qNh = P.qNh + (long long)jj * nx;
  auto Lz = [&](int e, T& Lo, T& Ln, T& Ld, T& Lrd) {
    long long idx;
    T g;
    if (e < nx) {
      g = ldr(qNh + e); idx = xo + e;
    } else {
      g = T(0.5); idx = is;
    }
    const T o = ldc(z + idx), nn = ldc(vout + idx);
    Lo = g * o; Ln = g * nn; Ld = g * (o - nn); Lrd = g * dirv(vref, idx);
  };
  soc_block<T, NE>(P, lane, nx + 2, P.e_qN + (long long)jj * (nx + 2), eta, eo, er, Lz, ra,
                   P.acostN ? P.acostN + (size_t)jj * (nx + 2) : nullptr);
}

// The soft-cost rows of non-leaf node i: [theta/s, sigma/2, sigma/2] in the
// translated cone SOC + (0, 1/2, -1/2), theta >= 0, theta - (x^i, u^i) >= lo.
template <class T, int NE>
__device__ void eta_soft(const Prob<T>& P, int lane, int i, const T* __restrict__ vin, T* __restrict__ vout,
                         const T* __restrict__ vref, RedAcc<T>& ra) {
  const int nx = P.nx, nu = P.nu, d = nx + nu;
  const T* z = vin;
  const T* eta = vin + P.nz;
  T* eo = vout + P.nz;
  const T* er = vref ? vref + P.nz : nullptr;
  const T al = P.alpha;
  const long long se = P.e_sf + (long long)i * (3 * d + 2);
  const long long ot = P.o_sth + (long long)i * d, isg = P.o_sg + i;
  // the cone through soc_block_vals (the instantiation the full-weight cost
  // cones already use: no second copy of the projection code)
  T ebv[NE], ldv[NE], lrv[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = lane + 32 * q;
    ebv[q] = T(0); ldv[q] = T(0); lrv[q] = T(0);
    if (e < d + 2) {
      long long idx;
      T g;
      if (e < d) { g = ldr(P.smw + e); idx = ot + e; }
      else { g = T(0.5); idx = isg; }
      const T o = ldc(z + idx), nn = ldc(vout + idx);
      ebv[q] = ldc(eta + se + e) + al * (T(2) * g * nn - g * o);
      ldv[q] = g * (o - nn);
      lrv[q] = g * dirv(vref, idx);
    }
  }
  soc_block_vals<T, NE>(P, lane, d + 2, se, eta, eo, er, ebv, ldv, lrv, nullptr, ra);
  auto row = [&](long long ie, T Lo, T Ln, T Ld, T Lrd, T lo) {
    const T eo_ = ldc(eta + ie);
    const T eb = eo_ + al * (T(2) * Ln - Lo);
    const T en = eta_prox(P, ie, eb, [&](auto w) { return max(w, (decltype(w))lo); });
    stc(eo + ie, en);
    ra.eta(eo_, en, er ? ldc(er + ie) : T(0), Ld, Lrd);
  };
  for (int k = lane; k < d; k += 32) {
    const T to = ldc(z + ot + k), tn = ldc(vout + ot + k), tr = dirv(vref, ot + k);
    const long long iz = (k < nx) ? P.o_x + (long long)i * nx + k : P.o_u + (long long)i * nu + (k - nx);
    const T zo = ldc(z + iz), zn = ldc(vout + iz), zr = dirv(vref, iz);
    row(se + d + 2 + k, to, tn, to - tn, tr, T(0));
    row(se + 2 * d + 2 + k, to - zo, tn - zn, (to - tn) - (zo - zn), tr - zr, ldr(P.slo + k));
  }
}

// ---------------------------------------------------------------------------
// shared memory views: per warp (phase P) and per team (phases B, F)
// ---------------------------------------------------------------------------
template <class T, int CH>
struct Views {
  static constexpr int D = Acc<T, CH>::D;
  T* base;
  int tw;
  // per warp: in, xb, red  (3 D)
  __device__ T* w_in(int w) const { return base + (size_t)w * 3 * D; }
  __device__ T* w_xb(int w) const { return base + (size_t)w * 3 * D + D; }
  __device__ T* w_red(int w) const { return base + (size_t)w * 3 * D + 2 * D; }
  // per team: in, xn, xb, qc, red (tw D); the two pipe buffers of every team
  // sit in front of `base` (see bytes()) so they never overlap any scratch
  size_t pipe_elems;   // elements of one pipe buffer (multiple of 16 bytes)
  T* pipe_base;
  __device__ T* t_base(int t) const { return base + (size_t)t * (4 + tw) * D; }
  __device__ T* t_pipe(int t, int b) const { return pipe_base + ((size_t)t * 2 + b) * pipe_elems; }
  __host__ __device__ static size_t pipe_elems_for(int pipe_bytes) {
    return (size_t)((pipe_bytes + 15) / 16) * 16 / sizeof(T);
  }
  // dynamic shared memory: the larger of the per-warp and per-team views; the
  // mbarriers live in a static array
  static size_t bytes(int threads, int tw, int pipe_bytes) {
    const int warps = threads / 32, teams = warps / tw;
    const size_t a = (size_t)warps * 3 * D;
    const size_t b = (size_t)teams * (4 + tw) * D;
    return ((a > b ? a : b) + (size_t)teams * 2 * pipe_elems_for(pipe_bytes)) * sizeof(T);
  }
};

// ---------------------------------------------------------------------------
// one evaluation of T: v_out = T(v_in); the reductions include the M-inner
// products of r = v_in - T(v_in) with the direction vref (none when null)
// ---------------------------------------------------------------------------
// Not inlined: the driver calls it from six places, and six inlined copies of
// the whole evaluation overflow the instruction cache.
template <class T, int CH>
__device__ __noinline__ bool evalT(const Prob<T>& P, const Team& tm, const Views<T, CH>& sv, Pipe<T>& pp,
                      CtaState& cs, int tg, int nt, const T* __restrict__ vin, T* __restrict__ vout,
                      const T* __restrict__ vref, double (&red)[NRED], double* partials,
                      SolveCtl* ctl, Grid& g) {
  constexpr int D = Acc<T, CH>::D;
  constexpr int NE = (D + 2 + 31) / 32;
  RedAcc<T> ra;
  ra.zero();
  PhaseClock pc;
  pc.start(g.prof);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = g.rank * (blockDim.x >> 5) + wid;
  const int nw = g.size * (blockDim.x >> 5);
  Team w1;
  w1.tw = 1; w1.id = wid; w1.warp = 0; w1.lane = lane; w1.tid = lane; w1.nth = 32;
  bool team_issued = false;   // the team path's first bulk copy is in flight
  if (P.cta) {
    ++cs.epoch;
    if (P.n_levels > 0 && seg_count(P, 0, tg, nt) > 0)
      ring_prefetch(P, cs.ring, seg_get(P, *cs.sched, 0, 0, tg, nt), false);
  } else if (pp.on && P.n_levels > 0) {
    const int s0 = P.lvl_off[0] + tg;
    if (s0 < P.lvl_off[1]) {
      issue_first_B<T, CH>(P, tm, pp, s0);
      team_issued = true;
    }
  }
    // P
  for (int node = gw; node < P.n; node += nw) {
    if (node < P.n_nl)
      prep_nonleaf<T, CH>(P, w1, sv.w_in(wid), sv.w_xb(wid), sv.w_red(wid), node, vin, vout, vref, ra);
    else
      prep_leaf(P, lane, node, vin);
    __syncwarp();
  }
  if (!grid_sync(g)) {
    // the launch is failing: let the copies issued before phase P land
    // (bounded) so that no bulk copy into this CTA's shared memory outlives it
    if (P.cta) {
      ring_settle(cs.ring, cs.ring.ahead);
    } else {
      if (team_issued && tm.tid == 0) {
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(pp.bar + pp.cur, pp.par[pp.cur]) && global_ns() - t0 < 200000000ull) {
        }
      }
      __syncthreads();
    }
    return false;
  }
  pc.mark(ctl, 0);
  // B
  const int L = P.n_levels;
  if (P.cta) {
    const Sched& S = *cs.sched;
    for (int l = 0; l < L; ++l) {
      const int m = seg_count(P, l, tg, nt);
      for (int k = 0; k < m; ++k) {
        const SegRef sr = seg_get(P, S, l, k, tg, nt);
        if (!bwd_cta<T>(P, cs.mem, cs.ring, &g.ctl->error, sr, cs.s_ok, g.prof, cs.seg_flags, 2u * cs.epoch))
          return false;
        // first items of this CTA's next segment (this level, a later one, or the first forward one)
        if (k + 1 < m) {
          ring_prefetch(P, cs.ring, seg_get(P, S, l, k + 1, tg, nt), false);
        } else {
          int l2 = l + 1;
          while (l2 < L && seg_count(P, l2, tg, nt) == 0) ++l2;
          if (l2 < L) ring_prefetch(P, cs.ring, seg_get(P, S, l2, 0, tg, nt), false);
          else if (seg_count(P, L - 1, tg, nt) > 0) ring_prefetch(P, cs.ring, seg_get(P, S, L - 1, 0, tg, nt), true);
          else {
            int l3 = L - 2;
            while (l3 >= 0 && seg_count(P, l3, tg, nt) == 0) --l3;
            if (l3 >= 0) ring_prefetch(P, cs.ring, seg_get(P, S, l3, 0, tg, nt), true);
          }
        }
      }
    }
    // no barrier between levels or before the forward sweep: segment flags order them
  } else {
    T* tb = sv.t_base(tm.id);
    for (int l = 0; l < L; ++l) {
      bool pre = pp.on;
      for (int s = P.lvl_off[l] + tg; s < P.lvl_off[l + 1]; s += nt) {
        const bool okb = backward_segment<T, CH>(P, tm, tb, tb + D, pp, &g.ctl->error, s, pre, g.prof);
        if (!okb) return false;
        pre = false;
      }
      if (pp.on) {   // first copy of this team's next piece of work, before the barrier
        if (l + 1 < L) {
          const int s1 = P.lvl_off[l + 1] + tg;
          if (s1 < P.lvl_off[l + 2]) issue_first_B<T, CH>(P, tm, pp, s1);
        } else {
          const int s1 = P.lvl_off[L - 1] + tg;
          if (s1 < P.lvl_off[L]) issue_first_F<T, CH>(P, tm, pp, s1);
        }
      }
      if (!grid_sync(g)) return false;
    }
  }
  pc.mark(ctl, 1);
  // F
  if (P.cta) {
    const Sched& S = *cs.sched;
    for (int l = L - 1; l >= 0; --l) {
      const int m = seg_count(P, l, tg, nt);
      for (int k = 0; k < m; ++k) {
        const SegRef sr = seg_get(P, S, l, k, tg, nt);
        if (!fwd_cta<T>(P, cs.mem, cs.ring, &g.ctl->error, sr, vout, cs.s_ok, g.prof, cs.seg_flags,
                        2u * cs.epoch + 1u))
          return false;
        if (k + 1 < m) {
          ring_prefetch(P, cs.ring, seg_get(P, S, l, k + 1, tg, nt), true);
        } else {
          int l2 = l - 1;
          while (l2 >= 0 && seg_count(P, l2, tg, nt) == 0) --l2;
          if (l2 >= 0) ring_prefetch(P, cs.ring, seg_get(P, S, l2, 0, tg, nt), true);
        }
      }
    }
    if (!grid_sync(g)) return false;   // phase E reads every node's x and u
  } else {
    T* tb = sv.t_base(tm.id);
    for (int l = L - 1; l >= 0; --l) {
      bool pre = pp.on;
      for (int s = P.lvl_off[l] + tg; s < P.lvl_off[l + 1]; s += nt) {
        const bool okf = forward_segment<T, CH>(P, tm, tb, tb + D, pp, &g.ctl->error, s, vout, pre);
        if (!okf) return false;
        pre = false;
      }
      if (pp.on && l > 0) {
        const int s1 = P.lvl_off[l - 1] + tg;
        if (s1 < P.lvl_off[l]) issue_first_F<T, CH>(P, tm, pp, s1);
      }
      if (!grid_sync(g)) return false;
    }
  }
  pc.mark(ctl, 2);
  // E
  {
    const long long nb = (long long)P.n_nl + (P.n - 1) + P.n_l;
    for (long long b = gw; b < nb; b += nw) {
      if (b < P.n_nl) {
        z_resid(vin, vout, vref, P.o_x + b * P.nx, P.nx, lane, ra);
        z_resid(vin, vout, vref, P.o_u + b * P.nu, P.nu, lane, ra);
        eta_nonleaf(P, lane, (int)b, vin, vout, vref, ra);
        if (P.l1 != T(0)) eta_l1(P, lane, (int)b, vin, vout, vref, ra);
        if (P.soft) eta_soft<T, NE>(P, lane, (int)b, vin, vout, vref, ra);
      } else if (b < P.n_nl + P.n - 1) {
        if (P.full) eta_soc_full<T, NE>(P, lane, (int)(b - P.n_nl + 1), vin, vout, vref, ra);
        else eta_soc<T, NE>(P, lane, (int)(b - P.n_nl + 1), vin, vout, vref, ra);
      } else {
        const int j = (int)(b - P.n_nl - (P.n - 1) + P.n_nl);
        z_resid(vin, vout, vref, P.o_x + (long long)j * P.nx, P.nx, lane, ra);
        eta_leaf<T, NE>(P, lane, j, vin, vout, vref, ra);
      }
    }
  }
  double v[NRED];
  __shared__ double scratch[NRED * 32];
  bool ok;
  // FP32 partials combined as float pairs in the one-chunk kernels; the
  // two-chunk FP32 kernel keeps the FP64 combine (with the pairs its team
  // sweeps ran about 20 % slower on the 498-node, nx = 128 problem)
  if constexpr (sizeof(T) == 4 && CH == 1) {
    DF dv[NRED];
#pragma unroll
    for (int k = 0; k < NRED; ++k) dv[k] = DF{ra.v[k], 0.0f};
    __shared__ double s_tot[NRED];
    ok = grid_allreduce_df(g, dv, v, reinterpret_cast<DF*>(scratch), s_tot, R_MAX);
  } else {
#pragma unroll
    for (int k = 0; k < NRED; ++k) v[k] = (double)ra.v[k];
    ok = grid_allreduce(g, v, scratch, R_MAX);
  }
#pragma unroll
  for (int k = 0; k < NRED; ++k) red[k] = v[k];
  pc.mark(ctl, 3);
  if (pc.on) g.prof[7] += 1;
  return ok;
}

// ---------------------------------------------------------------------------
// 16-byte vector load/store of the element-wise passes (L2 path)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void ldv(const T* p, long long q, T (&o)[Vec<T>::N]) {
  using V = typename Vec<T>::V;
  const V x = __ldcg(reinterpret_cast<const V*>(p) + q);
  memcpy(o, &x, sizeof(V));
}
template <class T>
__device__ __forceinline__ void stv(T* p, long long q, const T (&o)[Vec<T>::N]) {
  using V = typename Vec<T>::V;
  V x;
  memcpy(&x, o, sizeof(V));
  __stcg(reinterpret_cast<V*>(p) + q, x);
}

// kappa of the Anderson least-squares problem min ||Y kappa - r||_2 from the
// Gram matrix G = Y'Y (ring slots) and b = Y'r: Cholesky factorisation of G
// in the memory's logical order (oldest pair first, starting at ring slot
// `start`), the rank test on its pivots (a pivot R_jj below
// rank_tol * sqrt(trace G) = rank_tol * ||Y||_F rejects the direction), then
// the two triangular solves. Every index is fixed at compile time (the ring
// rotation and the unused slots are selects), so it runs in registers; one
// thread calls it, because FP64 arithmetic is slow on this part and 256
// redundant copies cost as much as the Anderson pass itself. Slots j >= count
// take an identity row, which gives kappa_j = 0. Returns false when the test
// rejects; kap is in ring-slot order.
__device__ __forceinline__ bool aa_gram_kappa(const double (&G)[AA_M][AA_M], const double (&b)[AA_M], int count,
                                              int start, double rank_tol, double (&kap)[AA_M]) {
  static_assert(AA_M == 3, "aa_gram_kappa is written for a memory of three pairs");
  double g[3][3], bl[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const double v = (start == 0) ? G[j][l] : ((start == 1) ? G[(j + 1) % 3][(l + 1) % 3] : G[(j + 2) % 3][(l + 2) % 3]);
      g[j][l] = (j < count && l < count) ? v : (j == l ? 1.0 : 0.0);
    }
    const double bv = (start == 0) ? b[j] : ((start == 1) ? b[(j + 1) % 3] : b[(j + 2) % 3]);
    bl[j] = (j < count) ? bv : 0.0;
  }
  double tr = g[0][0];
  if (count > 1) tr += g[1][1];
  if (count > 2) tr += g[2][2];
  if (!(tr > 0.0)) return false;
  const double lim2 = rank_tol * rank_tol * tr;   // R_jj < rank_tol sqrt(tr)  <=>  R_jj^2 < lim2
  const double d0 = g[0][0];
  if (!(d0 > 0.0) || d0 < lim2) return false;
  const double i0 = rsqrt(d0);
  const double r01 = g[0][1] * i0, r02 = g[0][2] * i0;
  const double d1 = fma(-r01, r01, g[1][1]);
  if (count > 1 && (!(d1 > 0.0) || d1 < lim2)) return false;
  const double i1 = rsqrt(d1);
  const double r12 = fma(-r01, r02, g[1][2]) * i1;
  const double d2 = fma(-r12, r12, fma(-r02, r02, g[2][2]));
  if (count > 2 && (!(d2 > 0.0) || d2 < lim2)) return false;
  const double i2 = rsqrt(d2);
  // R'c = b, then R k = c
  const double c0 = bl[0] * i0;
  const double c1 = fma(-r01, c0, bl[1]) * i1;
  const double c2 = fma(-r12, c1, fma(-r02, c0, bl[2])) * i2;
  const double k2 = c2 * i2;
  const double k1 = fma(-r12, k2, c1) * i1;
  const double k0 = fma(-r02, k2, fma(-r01, k1, c0)) * i0;
  const double kl[3] = {k0, k1, k2};
#pragma unroll
  for (int p = 0; p < 3; ++p)
    kap[p] = (start == 0) ? kl[p] : ((start == 1) ? kl[(p + 2) % 3] : kl[(p + 1) % 3]);
  return true;
}

// Anderson memory with the least-squares factorisation Y = Q R kept up to
// date (the improvement suggested in Sec. 6.2): pass A writes the new pair's s
// into the S ring, parks y = r - r_prev in PSI and reduces Q'y, Q'r and y'r;
// when the memory is full the oldest column is dropped by two Givens
// rotations of R's rows (applied to Q's columns in pass B); pass B appends
// w = y - Q h, h = Q'y (classical Gram-Schmidt), and reduces ||w||^2. Every
// CTA then holds R (3 x 3, FP64) and g = Q'r; kappa = R^{-1} g, and the
// direction is psi = -r - S kappa + Q g. Returns false when the launch fails.
template <class T>
__device__ bool aa_qr_update(const Prob<T>& P, const SolveBufs<T>& B, const SolveOpts& o, Grid& g, int k,
                             const T* V, const T* TV, int& head, int& count, double (&Rq)[AA_M][AA_M],
                             double (&qsc)[AA_M], int& qcount, double (&kap)[AA_M], double (&kapY)[AA_M],
                             bool& use_aa) {
  constexpr int VN = Vec<T>::N;
  const long long nv = P.nv, nvec = nv / VN, ss = B.sstride;
  const long long gtid = (long long)g.rank * blockDim.x + threadIdx.x;
  const long long gstride = (long long)g.size * blockDim.x;
  const bool push = k >= 1;
  const int slot = head;
  T* Sslot = B.S + slot * ss;
  // pass A
  double acc[NRED];
#pragma unroll
  for (int a = 0; a < NRED; ++a) acc[a] = 0.0;
  auto elemA = [&](T v, T tv, T vp, T rp, T q0, T q1, T q2, T& so, T& yo, T& ro) {
    const T r = v - tv;
    ro = r;
    so = v - vp;
    const T y = r - rp;
    yo = y;
    const T ql[AA_M] = {q0, q1, q2};
#pragma unroll
    for (int l = 0; l < AA_M; ++l) {
      acc[l] = fma((double)ql[l], (double)y, acc[l]);
      acc[AA_M + l] = fma((double)ql[l], (double)r, acc[AA_M + l]);
    }
    acc[2 * AA_M] = fma((double)y, (double)r, acc[2 * AA_M]);
  };
  for (long long q = gtid; q < nvec; q += gstride) {
    T v[VN], tv[VN], vp[VN], rp[VN], q0[VN], q1[VN], q2[VN], so[VN], yo[VN], ro[VN];
    ldv(V, q, v); ldv(TV, q, tv);
    if (push) {
      ldv((const T*)B.VP, q, vp); ldv((const T*)B.RP, q, rp);
      ldv((const T*)B.Y, q, q0); ldv((const T*)B.Y + ss, q, q1); ldv((const T*)B.Y + 2 * ss, q, q2);
#pragma unroll
      for (int c = 0; c < VN; ++c) elemA(v[c], tv[c], vp[c], rp[c], q0[c], q1[c], q2[c], so[c], yo[c], ro[c]);
      stv(Sslot, q, so); stv(B.PSI, q, yo);
    } else {
#pragma unroll
      for (int c = 0; c < VN; ++c) ro[c] = v[c] - tv[c];
    }
    stv(B.VP, q, v); stv(B.RP, q, ro);
  }
  for (long long e = nvec * VN + gtid; e < nv; e += gstride) {
    const T v = ldc(V + e), tv = ldc(TV + e);
    T so, yo, ro = v - tv;
    if (push) {
      elemA(v, tv, ldc(B.VP + e), ldc(B.RP + e), ldc(B.Y + e), ldc(B.Y + ss + e), ldc(B.Y + 2 * ss + e), so, yo, ro);
      stc(Sslot + e, so);
      stc(B.PSI + e, yo);
    }
    stc(B.VP + e, v);
    stc(B.RP + e, ro);
  }
  {
    __shared__ double scr[NRED * 32];
    if (!grid_allreduce(g, acc, scr, -1)) return false;
  }
  if (!push) return true;
  double hy[AA_M], hr[AA_M];
  for (int l = 0; l < AA_M; ++l) {
    hy[l] = l < qcount ? acc[l] * qsc[l] : 0.0;
    hr[l] = l < qcount ? acc[AA_M + l] * qsc[l] : 0.0;
  }
  const double yr = acc[2 * AA_M];
  // new basis b_j = sum_i cm[j][i] slot_i for the kept columns
  double cm[AA_M][AA_M];
  for (int a = 0; a < AA_M; ++a) for (int b = 0; b < AA_M; ++b) cm[a][b] = (a == b && a < qcount) ? qsc[a] : 0.0;
  int kept = qcount;
  if (qcount == AA_M) {   // drop the oldest column: R[:, 1:] is Hessenberg, two rotations
    double H[AA_M][AA_M - 1];
    for (int a = 0; a < AA_M; ++a) for (int b = 0; b < AA_M - 1; ++b) H[a][b] = Rq[a][b + 1];
    double rot[AA_M][AA_M];   // rows of the product of rotations (applied to Q's columns)
    for (int a = 0; a < AA_M; ++a) for (int b = 0; b < AA_M; ++b) rot[a][b] = (a == b) ? 1.0 : 0.0;
    for (int j = 0; j < AA_M - 1; ++j) {
      const double a = H[j][j], b = H[j + 1][j];
      const double r = hypot(a, b);
      const double c = r == 0.0 ? 1.0 : a / r, sn = r == 0.0 ? 0.0 : b / r;
      for (int q = 0; q < AA_M - 1; ++q) {
        const double x0 = H[j][q], x1 = H[j + 1][q];
        H[j][q] = c * x0 + sn * x1;
        H[j + 1][q] = -sn * x0 + c * x1;
      }
      for (int q = 0; q < AA_M; ++q) {
        const double x0 = rot[j][q], x1 = rot[j + 1][q];
        rot[j][q] = c * x0 + sn * x1;
        rot[j + 1][q] = -sn * x0 + c * x1;
      }
    }
    kept = AA_M - 1;
    for (int a = 0; a < AA_M; ++a) for (int b = 0; b < AA_M; ++b) Rq[a][b] = 0.0;
    for (int a = 0; a < kept; ++a) for (int b = a; b < kept; ++b) Rq[a][b] = H[a][b];
    double hy2[AA_M] = {0.0, 0.0, 0.0}, hr2[AA_M] = {0.0, 0.0, 0.0};
    for (int a = 0; a < kept; ++a)
      for (int b = 0; b < AA_M; ++b) {
        cm[a][b] = rot[a][b] * qsc[b];
        hy2[a] += rot[a][b] * hy[b];
        hr2[a] += rot[a][b] * hr[b];
      }
    for (int b = 0; b < AA_M; ++b) cm[kept][b] = 0.0;
    for (int a = 0; a < AA_M; ++a) { hy[a] = hy2[a]; hr[a] = hr2[a]; }
  }
  // pass B: rotated basis and w = y - sum_j hy_j b_j into slot `kept`
  const T c00 = (T)cm[0][0], c01 = (T)cm[0][1], c02 = (T)cm[0][2];
  const T c10 = (T)cm[1][0], c11 = (T)cm[1][1], c12 = (T)cm[1][2];
  const T h0 = (T)hy[0], h1 = (T)hy[1];
  double wacc[NRED];
#pragma unroll
  for (int a = 0; a < NRED; ++a) wacc[a] = 0.0;
  T* Yk = B.Y + kept * ss;
  auto elemB = [&](T q0, T q1, T q2, T y, T& b0, T& b1, T& w) {
    b0 = kept > 0 ? c00 * q0 + c01 * q1 + c02 * q2 : T(0);
    b1 = kept > 1 ? c10 * q0 + c11 * q1 + c12 * q2 : T(0);
    w = y - h0 * b0 - h1 * b1;
    wacc[0] = fma((double)w, (double)w, wacc[0]);
  };
  for (long long q = gtid; q < nvec; q += gstride) {
    T q0[VN], q1[VN], q2[VN], y[VN], b0[VN], b1[VN], w[VN];
    ldv((const T*)B.Y, q, q0); ldv((const T*)B.Y + ss, q, q1); ldv((const T*)B.Y + 2 * ss, q, q2);
    ldv((const T*)B.PSI, q, y);
#pragma unroll
    for (int c = 0; c < VN; ++c) elemB(q0[c], q1[c], q2[c], y[c], b0[c], b1[c], w[c]);
    if (kept > 0) stv(B.Y, q, b0);
    if (kept > 1) stv(B.Y + ss, q, b1);
    stv(Yk, q, w);
  }
  for (long long e = nvec * VN + gtid; e < nv; e += gstride) {
    T b0, b1, w;
    elemB(ldc(B.Y + e), ldc(B.Y + ss + e), ldc(B.Y + 2 * ss + e), ldc(B.PSI + e), b0, b1, w);
    if (kept > 0) stc(B.Y + e, b0);
    if (kept > 1) stc(B.Y + ss + e, b1);
    stc(Yk + e, w);
  }
  {
    __shared__ double scr2[NRED * 32];
    if (!grid_allreduce(g, wacc, scr2, -1)) return false;
  }
  const double rho = sqrt(fmax(wacc[0], 0.0));
  for (int a = 0; a < kept; ++a) { Rq[a][kept] = hy[a]; qsc[a] = 1.0; }
  Rq[kept][kept] = rho;
  qsc[kept] = rho > 0.0 ? 1.0 / rho : 0.0;
  qcount = kept + 1;
  // Q'r in the new basis: w'r / rho = (y'r - h . hr) / rho
  double gq[AA_M] = {0.0, 0.0, 0.0};
  for (int a = 0; a < kept; ++a) gq[a] = hr[a];
  {
    double wr = yr;
    for (int a = 0; a < kept; ++a) wr -= hy[a] * hr[a];
    gq[kept] = rho > 0.0 ? wr / rho : 0.0;
  }
  if (count < AA_M) ++count;
  head = (head + 1) % AA_M;
  if (k > AA_M && qcount > 0) {
    double fro = 0.0;
    for (int a = 0; a < qcount; ++a) for (int b = a; b < qcount; ++b) fro += Rq[a][b] * Rq[a][b];
    fro = sqrt(fro);
    bool good = fro > 0.0;
    for (int a = 0; a < qcount && good; ++a) good = fabs(Rq[a][a]) >= o.rank_tol * fro;
    if (good) {
      double kl[AA_M];
      for (int j = qcount - 1; j >= 0; --j) {
        double sacc = gq[j];
        for (int l = j + 1; l < qcount; ++l) sacc -= Rq[j][l] * kl[l];
        kl[j] = sacc / Rq[j][j];
      }
      // logical column j of Q pairs with the j-th oldest s in the S ring
      const int start = (count < AA_M) ? 0 : head;
      for (int j = 0; j < qcount; ++j) {
        kap[(start + j) % AA_M] = kl[j];
        kapY[j] = gq[j] * qsc[j];
      }
      use_aa = true;
    }
  }
  return true;
}

// The SuperMann iteration (Alg. 4 with Anderson directions, Alg. 3) on one
// problem by the group g: the whole grid of a single-problem launch, or one
// CTA of the batched launch. Every CTA of the group runs the same scalar
// control flow on the group-reduced scalars.
template <class T, int CH>
__device__ void solve_loop(const Prob<T>& P, const SolveBufs<T>& B, const SolveOpts& o, const Team& tm,
                           const Views<T, CH>& sv, Pipe<T>& pp, CtaState& cs, int tg, int nt, Grid& g) {
  SolveCtl* ctl = B.ctl;
  T* buf[4] = {B.V, B.TV, B.VT, B.TVT};
  int iV = 0, iTV = 1, iVT = 2, iTVT = 3;
  const long long nv = P.nv;
  const long long gtid = (long long)g.rank * blockDim.x + threadIdx.x;
  const long long gstride = (long long)g.size * blockDim.x;
  constexpr int VN = Vec<T>::N;
  const long long nvec = nv / VN;
  const long long ss = B.sstride;
  const T al = P.alpha;
  double red[NRED];
  int status = 0, k = 0, nT = 0, nK0 = 0, nK1 = 0, nK2 = 0, nFB = 0, nBT = 0;
  double res, om2;
  bool ok = evalT<T, CH>(P, tm, sv, pp, cs, tg, nt, buf[iV], buf[iTV], (const T*)nullptr, red, B.partials, ctl, g);
  ++nT;
  if (!ok) goto fail;
  res = red[R_MAX];
  om2 = red[R_ZZ] + red[R_EE] - 2.0 * (double)al * red[R_ELZ];
  if (o.method == 2) goto done;
  if (o.method == 1) {
    while (!(res <= o.tol) && k < o.max_iters) {
      int t = iV; iV = iTV; iTV = t;
      ok = evalT<T, CH>(P, tm, sv, pp, cs, tg, nt, buf[iV], buf[iTV], (const T*)nullptr, red, B.partials, ctl, g);
      ++nT; ++k;
      if (!ok) goto fail;
      res = red[R_MAX];
      om2 = red[R_ZZ] + red[R_EE] - 2.0 * (double)al * red[R_ELZ];
    }
    status = (res <= o.tol) ? 0 : 1;
    goto done;
  }
  {
    double zeta = sqrt(fmax(om2, 0.0)), omega_safe = zeta;
    double G[AA_M][AA_M];
    for (int a = 0; a < AA_M; ++a) for (int b = 0; b < AA_M; ++b) G[a][b] = 0.0;
    int count = 0, head = 0;
    // updated-QR mode: Y = Q R with the columns of Q in the Y slots in logical
    // order (oldest first), slot j holding Q's column j divided by qsc[j]
    double Rq[AA_M][AA_M], qsc[AA_M];
    for (int a = 0; a < AA_M; ++a) { qsc[a] = 1.0; for (int b = 0; b < AA_M; ++b) Rq[a][b] = 0.0; }
    int qcount = 0;
    while (true) {
      if (res <= o.tol) { status = 0; break; }
      if (k >= o.max_iters) { status = 1; break; }
      const double omega = sqrt(fmax(om2, 0.0));
      T* V = buf[iV];
      T* TV = buf[iTV];
      PhaseClock pc;
      pc.start(g.prof);
      // --- Anderson memory update (pairs (v^k - v^{k-1}, r^k - r^{k-1})) ---
      double kap[AA_M] = {0.0, 0.0, 0.0};    // coefficients of the S slots
      double kapY[AA_M] = {0.0, 0.0, 0.0};   // coefficients of the Y slots
      bool use_aa = false;
      if (o.aa_qr) {
        if (!aa_qr_update<T>(P, B, o, g, k, V, TV, head, count, Rq, qsc, qcount, kap, kapY, use_aa)) goto fail;
      } else {
        const int slot = head;
        const bool push = (k >= 1);
        double dd[NRED];
        // the Gram matrix Y'Y and Y'r are accumulated to FP64 accuracy in
        // every precision: their condition is the square of Y's
        double acc[2 * AA_M];
        for (int a = 0; a < 2 * AA_M; ++a) acc[a] = 0.0;
        // FP32: the same sums in compensated single precision (the dot product
        // of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005: the
        // exact product p + ep by an FMA, the running sum hi + lo by an
        // error-free two-sum), as accurate as an FP64 accumulation of the FP32
        // products but on the FP32 pipe -- B300's FP64 pipe issues about 1/77
        // of the FP32 rate
        float chi[2 * AA_M], clo[2 * AA_M];
        for (int a = 0; a < 2 * AA_M; ++a) { chi[a] = 0.0f; clo[a] = 0.0f; }
        // (the _rn intrinsics keep the compiler from contracting the
        // transformation's products and sums into FMAs)
        auto dot2 = [&](int a, float x, float y) {
          const float pr = __fmul_rn(x, y);
          const float ep = fmaf(x, y, -pr);
          const float sm = __fadd_rn(chi[a], pr);
          const float bb = __fsub_rn(sm, chi[a]);
          const float es = __fadd_rn(__fsub_rn(chi[a], __fsub_rn(sm, bb)), __fsub_rn(pr, bb));
          chi[a] = sm;
          clo[a] = __fadd_rn(clo[a], __fadd_rn(ep, es));
        };
        T* Sslot = B.S + slot * ss;
        T* Yslot = B.Y + slot * ss;
        // one element: new pair (s, y), dots y.Y_l and Y_l.r, copies of v and r
        auto elem = [&](T v, T tv, T vp, T rp, T y0, T y1, T y2, T& so, T& yo, T& ro) {
          const T r = v - tv;
          ro = r;
          so = v - vp;
          const T y_ = r - rp;
          yo = y_;
          const T yl[AA_M] = {slot == 0 ? y_ : y0, slot == 1 ? y_ : y1, slot == 2 ? y_ : y2};
#pragma unroll
          for (int l = 0; l < AA_M; ++l) {
            if constexpr (sizeof(T) == 4) {
              dot2(l, y_, yl[l]);
              dot2(AA_M + l, yl[l], r);
            } else {
              acc[l] = fma((double)y_, (double)yl[l], acc[l]);
              acc[AA_M + l] = fma((double)yl[l], (double)r, acc[AA_M + l]);
            }
          }
        };
        for (long long q = gtid; q < nvec; q += gstride) {
          T v[VN], tv[VN], vp[VN], rp[VN], y0[VN], y1[VN], y2[VN], so[VN], yo[VN], ro[VN];
          ldv(V, q, v); ldv(TV, q, tv);
          if (push) {
            ldv((const T*)B.VP, q, vp); ldv((const T*)B.RP, q, rp);
            ldv((const T*)B.Y, q, y0); ldv((const T*)B.Y + ss, q, y1); ldv((const T*)B.Y + 2 * ss, q, y2);
#pragma unroll
            for (int c = 0; c < VN; ++c) elem(v[c], tv[c], vp[c], rp[c], y0[c], y1[c], y2[c], so[c], yo[c], ro[c]);
            stv(Sslot, q, so); stv(Yslot, q, yo);
          } else {
#pragma unroll
            for (int c = 0; c < VN; ++c) ro[c] = v[c] - tv[c];
          }
          stv(B.VP, q, v); stv(B.RP, q, ro);
        }
        for (long long e = nvec * VN + gtid; e < nv; e += gstride) {
          const T v = ldc(V + e), tv = ldc(TV + e);
          T so, yo, ro = v - tv;
          if (push) {
            elem(v, tv, ldc(B.VP + e), ldc(B.RP + e), ldc(B.Y + e), ldc(B.Y + ss + e),
                 ldc(B.Y + 2 * ss + e), so, yo, ro);
            stc(Sslot + e, so);
            stc(Yslot + e, yo);
          }
          stc(B.VP + e, v);
          stc(B.RP + e, ro);
        }
        {
          __shared__ double scratch2[NRED * 32];
          if constexpr (sizeof(T) == 4 && CH == 1) {   // the compensated sums enter as pairs (sum, error)
            DF df[NRED];
#pragma unroll
            for (int a = 0; a < NRED; ++a) df[a] = DF{0.0f, 0.0f};
#pragma unroll
            for (int a = 0; a < 2 * AA_M; ++a) df[a] = DF{chi[a], clo[a]};
            __shared__ double s_tot2[NRED];
            if (!grid_allreduce_df(g, df, dd, reinterpret_cast<DF*>(scratch2), s_tot2, -1)) goto fail;
          } else {
            if constexpr (sizeof(T) == 4) {
              for (int a = 0; a < 2 * AA_M; ++a) acc[a] = (double)chi[a] + (double)clo[a];
            }
            for (int a = 0; a < NRED; ++a) dd[a] = (a < 2 * AA_M) ? acc[a] : 0.0;
            if (!grid_allreduce(g, dd, scratch2, -1)) goto fail;
          }
        }
        if (push) {
          if (count < AA_M) ++count;
          head = (head + 1) % AA_M;
#pragma unroll
          for (int a = 0; a < AA_M; ++a)
#pragma unroll
            for (int b = 0; b < AA_M; ++b) {
              if (a == slot) G[a][b] = dd[b];
              else if (b == slot) G[a][b] = dd[a];
            }
        }
        if (k > AA_M && count > 0) {
          __shared__ double s_kap[AA_M + 1];
          if (threadIdx.x == 0) {
            const double bvec[AA_M] = {dd[AA_M], dd[AA_M + 1], dd[AA_M + 2]};
            double kl[AA_M];
            const bool good = aa_gram_kappa(G, bvec, count, (count < AA_M) ? 0 : head, o.rank_tol, kl);
#pragma unroll
            for (int j = 0; j < AA_M; ++j) s_kap[j] = kl[j];
            s_kap[AA_M] = good ? 1.0 : 0.0;
          }
          __syncthreads();
          if (s_kap[AA_M] != 0.0) {
#pragma unroll
            for (int j = 0; j < AA_M; ++j) { kap[j] = s_kap[j]; kapY[j] = s_kap[j]; }
            use_aa = true;
          }
        }
      }
      pc.mark(ctl, 4);
      // --- psi and the first trial point v~ = v + psi ---
      {
        T* VT = buf[iVT];
        const T k0 = (T)kap[0], k1 = (T)kap[1], k2 = (T)kap[2];
        const T j0 = (T)kapY[0], j1 = (T)kapY[1], j2 = (T)kapY[2];
        auto elem = [&](T v, T tv, T s0, T s1, T s2, T y0, T y1, T y2, T& psi, T& vt) {
          T p = -(v - tv);
          if (use_aa) {   // psi = -r - S kappa + Y kappaY (kappaY = kappa, or Q'r in the QR mode)
            p -= s0 * k0 - y0 * j0;
            p -= s1 * k1 - y1 * j1;
            p -= s2 * k2 - y2 * j2;
          }
          psi = p;
          vt = v + p;
        };
        for (long long q = gtid; q < nvec; q += gstride) {
          T v[VN], tv[VN], s0[VN], s1[VN], s2[VN], y0[VN], y1[VN], y2[VN], ps[VN], vt[VN];
          ldv((const T*)V, q, v); ldv((const T*)TV, q, tv);
          if (use_aa) {
            ldv((const T*)B.S, q, s0); ldv((const T*)B.S + ss, q, s1); ldv((const T*)B.S + 2 * ss, q, s2);
            ldv((const T*)B.Y, q, y0); ldv((const T*)B.Y + ss, q, y1); ldv((const T*)B.Y + 2 * ss, q, y2);
          } else {
#pragma unroll
            for (int c = 0; c < VN; ++c) s0[c] = s1[c] = s2[c] = y0[c] = y1[c] = y2[c] = T(0);
          }
#pragma unroll
          for (int c = 0; c < VN; ++c) elem(v[c], tv[c], s0[c], s1[c], s2[c], y0[c], y1[c], y2[c], ps[c], vt[c]);
          stv(B.PSI, q, ps);
          stv(VT, q, vt);
        }
        for (long long e = nvec * VN + gtid; e < nv; e += gstride) {
          T ps, vt;
          const bool u = use_aa;
          elem(ldc(V + e), ldc(TV + e), u ? ldc(B.S + e) : T(0), u ? ldc(B.S + ss + e) : T(0),
               u ? ldc(B.S + 2 * ss + e) : T(0), u ? ldc(B.Y + e) : T(0), u ? ldc(B.Y + ss + e) : T(0),
               u ? ldc(B.Y + 2 * ss + e) : T(0), ps, vt);
          stc(B.PSI + e, ps);
          stc(VT + e, vt);
        }
      }
      if (!grid_sync(g)) goto fail;
      pc.mark(ctl, 5);
      ok = evalT<T, CH>(P, tm, sv, pp, cs, tg, nt, buf[iVT], buf[iTVT], B.PSI, red, B.partials, ctl, g);
      ++nT;
      if (!ok) goto fail;
      if (omega <= C0 * zeta) {                       // K0
        int t = iV; iV = iVT; iVT = t;
        t = iTV; iTV = iTVT; iTVT = t;
        zeta = omega;
        res = red[R_MAX];
        om2 = red[R_ZZ] + red[R_EE] - 2.0 * (double)al * red[R_ELZ];
        ++nK0; ++k;
        continue;
      }
      double tau = 1.0;
      int bt = 0;
      while (true) {
        const double om2t = red[R_ZZ] + red[R_EE] - 2.0 * (double)al * red[R_ELZ];
        const double omt = sqrt(fmax(om2t, 0.0));
        if ((omega <= omega_safe && omt <= C1 * omega) || omt == 0.0) {   // K1
          int t = iV; iV = iVT; iVT = t;
          t = iTV; iTV = iTVT; iTVT = t;
          omega_safe = omt + pow(C2, (double)k);
          res = red[R_MAX];
          om2 = om2t;
          ++nK1;
          break;
        }
        // <r~, v~ - v>_M with v~ - v = tau psi (psi as stored, not recovered by a subtraction)
        const double mdot = tau * (red[R_ZD] + red[R_ED] - (double)al * red[R_LZD] - (double)al * red[R_ELD]);
        const double rho = om2t - mdot;
        PhaseClock pk;
        pk.start(g.prof);
        if (rho >= SIGMA * omt * omega) {             // K2
          const T coef = (T)(LAMBDA * rho / om2t);
          T* Vc = buf[iV];
          T* VT = buf[iVT];
          const T* TVT = buf[iTVT];
          for (long long q = gtid; q < nvec; q += gstride) {
            T a[VN], b[VN], c_[VN];
            ldv((const T*)Vc, q, a); ldv((const T*)VT, q, b); ldv(TVT, q, c_);
#pragma unroll
            for (int c = 0; c < VN; ++c) b[c] = a[c] - coef * (b[c] - c_[c]);
            stv(VT, q, b);
          }
          for (long long e = nvec * VN + gtid; e < nv; e += gstride) {
            const T vt = ldc(VT + e);
            stc(VT + e, ldc(Vc + e) - coef * (vt - ldc(TVT + e)));
          }
          if (!grid_sync(g)) goto fail;
          pk.mark(ctl, 6);
          int t = iV; iV = iVT; iVT = t;
          ok = evalT<T, CH>(P, tm, sv, pp, cs, tg, nt, buf[iV], buf[iTV], (const T*)nullptr, red, B.partials, ctl, g);
          ++nT;
          if (!ok) goto fail;
          res = red[R_MAX];
          om2 = red[R_ZZ] + red[R_EE] - 2.0 * (double)al * red[R_ELZ];
          ++nK2;
          break;
        }
        ++bt; ++nBT;
        if (bt >= o.max_backtracks) {                 // fall back to v <- T(v)
          int t = iV; iV = iTV; iTV = t;
          ok = evalT<T, CH>(P, tm, sv, pp, cs, tg, nt, buf[iV], buf[iTV], (const T*)nullptr, red, B.partials, ctl, g);
          ++nT;
          if (!ok) goto fail;
          res = red[R_MAX];
          om2 = red[R_ZZ] + red[R_EE] - 2.0 * (double)al * red[R_ELZ];
          ++nFB;
          break;
        }
        tau *= BETA;
        {
          const T tt = (T)tau;
          const T* Vc = buf[iV];
          T* VT = buf[iVT];
          for (long long q = gtid; q < nvec; q += gstride) {
            T a[VN], b[VN];
            ldv(Vc, q, a); ldv((const T*)B.PSI, q, b);
#pragma unroll
            for (int c = 0; c < VN; ++c) a[c] = a[c] + tt * b[c];
            stv(VT, q, a);
          }
          for (long long e = nvec * VN + gtid; e < nv; e += gstride) stc(VT + e, ldc(Vc + e) + tt * ldc(B.PSI + e));
        }
        if (!grid_sync(g)) goto fail;
        pk.mark(ctl, 6);
        ok = evalT<T, CH>(P, tm, sv, pp, cs, tg, nt, buf[iVT], buf[iTVT], B.PSI, red, B.partials, ctl, g);
        ++nT;
        if (!ok) goto fail;
      }
      ++k;
    }
  }
done:
  if (g.rank == 0 && threadIdx.x == 0) {
    ctl->status = status;
    ctl->iters = k; ctl->n_T = nT; ctl->n_K0 = nK0; ctl->n_K1 = nK1; ctl->n_K2 = nK2;
    ctl->n_fb = nFB; ctl->n_bt = nBT;
    ctl->res_inf = res;
    for (int q = 0; q < NRED; ++q) ctl->stats[q] = red[q];
    ctl->final_v = iV;       // final buffer indices for the host
    ctl->final_tv = iTV;
    for (int q = 0; q < 16; ++q) ctl->prof[q] = g.prof[q];
  }
  return;
fail:
  if (g.rank == 0 && threadIdx.x == 0) {
    ctl->status = -5;
    ctl->iters = k; ctl->n_T = nT;
    ctl->final_v = iV;
    ctl->final_tv = iTV;
  }
}

// ---------------------------------------------------------------------------
// the solve kernel
// ---------------------------------------------------------------------------
template <class T, int CH>
__global__ void __launch_bounds__(256, 1) k_solve(Prob<T> Pk, SolveBufs<T> B, SolveOpts o, int tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // the problem descriptor lives in shared memory so that the non-inlined
  // evaluation reads it without a local-memory copy of the parameter
  __shared__ __align__(16) unsigned char s_prob[sizeof(Prob<T>)];
  for (int b = threadIdx.x; b < (int)sizeof(Prob<T>); b += blockDim.x)
    s_prob[b] = reinterpret_cast<const unsigned char*>(&Pk)[b];
  __syncthreads();
  const Prob<T>& P = *reinterpret_cast<const Prob<T>*>(s_prob);
  const Team tm = make_team(tw);
  const int teams_per_cta = (blockDim.x >> 5) / tw;
  const int tg = blockIdx.x * teams_per_cta + tm.id;
  const int nt = gridDim.x * teams_per_cta;
  Views<T, CH> sv;
  sv.tw = tw;
  sv.pipe_elems = Views<T, CH>::pipe_elems_for(P.pipe_bytes);
  const size_t cta_bytes = cta_smem_bytes(P);
  sv.pipe_base = reinterpret_cast<T*>(smraw + cta_bytes);
  sv.base = sv.pipe_base + (size_t)teams_per_cta * 2 * sv.pipe_elems;
  __shared__ __align__(8) uint64_t s_bar[2 * MAXTW];
  Pipe<T> pp;
  pp.on = P.pipe_bytes > 0;
  pp.bar = s_bar + 2 * tm.id;
  pp.buf[0] = sv.t_pipe(tm.id, 0);
  pp.buf[1] = sv.t_pipe(tm.id, 1);
  pp.par[0] = pp.par[1] = 0u;
  pp.cur = 0;
  __shared__ int s_ok[MAXTW];
  pp.okp = s_ok + tm.id;
  pp.diag = B.ctl->diag;
  if (threadIdx.x < 2 * MAXTW) mbar_init(s_bar + threadIdx.x, 1);
  fence_mbar_init();
  __syncthreads();
  // whole-CTA sweeps: ring of item buffers, carry vectors, child inputs, schedule
  CtaState cs;
  __shared__ Sched s_sched;
  __shared__ int s_cta_ok;
  if (P.cta) {
    const unsigned base = smem_u32(smraw);
    cs.ring.bar0 = smem_u32(s_bar);
    cs.ring.buf0 = base;
    cs.ring.bstride = (unsigned)P.item_bytes;
    cs.ring.nbuf = P.nbuf;
    cs.ring.par = 0u;
    cs.ring.head = 0;
    cs.ring.ahead = 0;
    cs.ring.diag = B.ctl->diag;
    const unsigned ldcb = (unsigned)(P.ldc * sizeof(T));
    cs.mem.carry0 = base + (unsigned)P.nbuf * (unsigned)P.item_bytes;
    cs.mem.carry1 = cs.mem.carry0 + ldcb;
    cs.mem.qin = cs.mem.carry1 + ldcb;
    // padding rows of the vectors are read against zero coefficients: keep them finite
    T* vz = reinterpret_cast<T*>(smraw + (size_t)P.nbuf * P.item_bytes);
    for (int k = threadIdx.x; k < (2 + P.qslots) * P.ldc; k += blockDim.x) vz[k] = T(0);
    sched_build(P, s_sched, tg, nt);
    cs.sched = &s_sched;
    cs.s_ok = &s_cta_ok;
    cs.seg_flags = B.flags + P.seg_flag_off;
    cs.epoch = 0;
  }
  SolveCtl* ctl = B.ctl;
#ifdef SPOCK_CHECKED
  if (threadIdx.x == 0) { g_chk_err = &ctl->bar.error; g_chk_site = &ctl->check_site; }
  __syncthreads();
#endif
  Grid g;
  g.ctl = &ctl->bar;
  g.flags = B.flags;
  g.partials = B.partials;
  g.epoch = 0;
  g.rank = blockIdx.x;
  g.size = gridDim.x + o.phantom;   // phantom > 0 only in tests of the timeout path
  g.local = false;
  g.limit_ns = o.wait_ns ? o.wait_ns : BARRIER_LIMIT_NS;
  __shared__ unsigned long long s_prof[16];
  if (threadIdx.x < 16) s_prof[threadIdx.x] = 0ull;
  __syncthreads();
  g.prof = s_prof;
  solve_loop<T, CH>(P, B, o, tm, sv, pp, cs, tg, nt, g);
}

// ---------------------------------------------------------------------------
// Batched launch. A persistent grid in which
//  - the first CTAs form gangs (BatchPlan): gang k of size g solves its static
//    list of large problems one after the other, its CTAs iterating on each
//    problem together with barriers and reductions among the gang's CTAs;
//  - every other CTA, and every gang CTA once its list is done, takes small
//    problems from a queue (small_order, largest first) and solves each one
//    alone, with the barriers and reductions inside the CTA.
// tws[p]: warps per team of problem p's sweeps (picked by the autotuner);
// cycles[p]: clock cycles that the first CTA of the problem spent on it.
// ---------------------------------------------------------------------------

// a struct of 8-byte words read through L2 (never from a non-coherent line):
// for table entries the host may write while a persistent launch runs
template <class X>
__device__ __forceinline__ X ld_struct_cg(const X* p) {
  static_assert(sizeof(X) % 8 == 0, "8-byte words");
  X out;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&out);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(X) / 8); ++k) dst[k] = __ldcg(src + k);
  return out;
}

template <class T, int CH>
__device__ __forceinline__ void batch_one(const Prob<T>* __restrict__ probs, const SolveBufs<T>& B,
                                          const int* __restrict__ tws, const SolveOpts& o, int pi, Grid& g,
                                          unsigned char* smraw, unsigned char* s_prob, uint64_t* s_bar, int* s_ok,
                                          unsigned long long* s_prof, bool first, long long* cycles) {
  const long long t0 = clock64();
  for (int b = threadIdx.x; b < (int)sizeof(Prob<T>); b += blockDim.x)
    s_prob[b] = reinterpret_cast<const unsigned char*>(probs + pi)[b];
  if (threadIdx.x < 16) s_prof[threadIdx.x] = 0ull;
  // fresh mbarrier phases for this problem (every copy of the last one was waited for)
  if (!first && threadIdx.x < 2 * MAXTW) {
    mbar_inval(s_bar + threadIdx.x);
    mbar_init(s_bar + threadIdx.x, 1);
  }
  fence_mbar_init();
  __syncthreads();
  const Prob<T>& P = *reinterpret_cast<const Prob<T>*>(s_prob);
  const int tw = tws[pi];
  const Team tm = make_team(tw);
  const int teams = (blockDim.x >> 5) / tw;
  Views<T, CH> sv;
  sv.tw = tw;
  sv.pipe_elems = Views<T, CH>::pipe_elems_for(P.pipe_bytes);
  sv.pipe_base = reinterpret_cast<T*>(smraw);
  sv.base = sv.pipe_base + (size_t)teams * 2 * sv.pipe_elems;
  Pipe<T> pp;
  pp.on = P.pipe_bytes > 0;
  pp.bar = s_bar + 2 * tm.id;
  pp.buf[0] = sv.t_pipe(tm.id, 0);
  pp.buf[1] = sv.t_pipe(tm.id, 1);
  pp.par[0] = pp.par[1] = 0u;
  pp.cur = 0;
  pp.okp = s_ok + tm.id;
  pp.diag = B.ctl->diag;
  CtaState cs{};   // the whole-CTA sweeps are not used in the batch (P.cta == 0)
  g.ctl = &B.ctl->bar;
  g.prof = s_prof;
  solve_loop<T, CH>(P, B, o, tm, sv, pp, cs, g.rank * teams + tm.id, g.size * teams, g);
  __syncthreads();
  if (threadIdx.x == 0 && g.rank == 0 && cycles) cycles[pi] = clock64() - t0;
}

template <class T, int CH>
__global__ void __launch_bounds__(256, 1)
    k_batch(const Prob<T>* __restrict__ probs, const SolveBufs<T>* __restrict__ bufs,
            const int* __restrict__ tws, SolveOpts o, BatchPlan plan, long long* __restrict__ cycles) {
  extern __shared__ __align__(16) unsigned char smraw[];
#ifdef SPOCK_CHECKED
  if (threadIdx.x == 0) g_chk_err = nullptr;   // the checks cover the single-problem launch
#endif
  __shared__ __align__(16) unsigned char s_prob[sizeof(Prob<T>)];
  __shared__ __align__(8) uint64_t s_bar[2 * MAXTW];
  __shared__ int s_ok[MAXTW];
  __shared__ unsigned long long s_prof[16];
  __shared__ int s_q;
  if (threadIdx.x < 2 * MAXTW) mbar_init(s_bar + threadIdx.x, 1);
  fence_mbar_init();
  __syncthreads();
  bool first = true;
  if ((int)blockIdx.x < plan.n_gang_ctas) {
    const int k = plan.gang_of[blockIdx.x];
    const int start = plan.gang_start[k];
    Grid g;
    g.rank = blockIdx.x - start;
    g.size = plan.gang_size[k];
    g.local = g.size == 1;
    g.limit_ns = o.wait_ns ? o.wait_ns : BARRIER_LIMIT_NS;
    g.flags = plan.flags + start;
    g.partials = plan.partials + (size_t)2 * NRED * start;
    g.epoch = 0;
    for (int q = plan.list_off[k]; q < plan.list_off[k + 1]; ++q) {
      batch_one<T, CH>(probs, bufs[plan.list[q]], tws, o, plan.list[q], g, smraw, s_prob, s_bar, s_ok, s_prof, first,
                       cycles);
      first = false;
    }
  }
  Grid g;
  g.rank = 0;
  g.size = 1;
  g.local = true;
  g.limit_ns = BARRIER_LIMIT_NS;
  g.flags = nullptr;
  g.partials = nullptr;
  g.epoch = 0;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(plan.next, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= plan.n_small) break;
    const int pi = plan.small_order[q];
    batch_one<T, CH>(probs, bufs[pi], tws, o, pi, g, smraw, s_prob, s_bar, s_ok, s_prof, first, cycles);
    first = false;
  }
}

// ---------------------------------------------------------------------------
// Serving: a persistent grid whose CTAs claim requests from the ring in mapped
// host memory as they are published, so requests that arrive while others run
// start as soon as a CTA is free. Each request runs alone in its CTA (barriers
// and reductions inside it): its result does not depend on the other requests.
// Leaves when ctl->stop is raised or after idle_ns without a request (the host
// relaunches it on the next submission). The grid leaves together: a CTA
// leaves only when no CTA is solving and no request was claimed for idle_ns,
// so a request published later never finds only a few CTAs alive.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long ld_acquire_sys(const volatile long long* p) {
  long long v;
  asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <class T, int CH>
__global__ void __launch_bounds__(256, 1)
    k_serve(const Prob<T>* __restrict__ probs, const SolveBufs<T>* bufs,
            const int* __restrict__ tws, const ServeMeta<T>* __restrict__ meta, SolveOpts o,
            const ServeReq* ring, ServeRes* res, int cap, ServeCtl* ctl, ServeDev* dev,
            unsigned long long idle_ns) {
  extern __shared__ __align__(16) unsigned char smraw[];
#ifdef SPOCK_CHECKED
  if (threadIdx.x == 0) g_chk_err = nullptr;   // the checks cover the single-problem launch
#endif
  __shared__ __align__(16) unsigned char s_prob[sizeof(Prob<T>)];
  __shared__ __align__(8) uint64_t s_bar[2 * MAXTW];
  __shared__ int s_ok[MAXTW];
  __shared__ unsigned long long s_prof[16];
  __shared__ long long s_q;
  if (threadIdx.x < 2 * MAXTW) mbar_init(s_bar + threadIdx.x, 1);
  fence_mbar_init();
  __syncthreads();
  Grid g;
  g.rank = 0; g.size = 1; g.local = true; g.flags = nullptr; g.partials = nullptr; g.epoch = 0;
  g.limit_ns = BARRIER_LIMIT_NS;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) {
      // claim the next published request (bounded idle wait)
      long long q = -1;
      const uint64_t t0 = global_ns();
      for (;;) {
        if (ctl->stop) break;
        const long long h = *reinterpret_cast<volatile long long*>(&dev->head);
        const long long tl = ld_acquire_sys(&ctl->tail);
        if (h < tl) {
          if (atomicCAS(reinterpret_cast<unsigned long long*>(&dev->head), (unsigned long long)h,
                        (unsigned long long)(h + 1)) == (unsigned long long)h) {
            q = h;
            atomicAdd(&dev->busy, 1);
            atomicMax(&dev->last_ns, (unsigned long long)global_ns());
            break;
          }
          continue;
        }
        const uint64_t now = global_ns();
        const unsigned long long last = *reinterpret_cast<volatile unsigned long long*>(&dev->last_ns);
        const int busy = *reinterpret_cast<volatile int*>(&dev->busy);
        if (busy == 0 && now - (last > t0 ? last : t0) > idle_ns) break;
        __nanosleep(2000);
      }
      s_q = q;
    }
    __syncthreads();
    const long long q = s_q;
    __syncthreads();
    if (q < 0) break;
    const ServeReq* rq = ring + (q % cap);
    ServeRes* rs = res + (q % cap);
    __shared__ int s_plant, s_warm;
    __shared__ long long s_id;
    __shared__ unsigned long long s_t0;
    if (threadIdx.x == 0) {
      s_plant = *reinterpret_cast<const volatile int*>(&rq->plant);
      s_warm = *reinterpret_cast<const volatile int*>(&rq->warm);
      s_id = *reinterpret_cast<const volatile long long*>(&rq->id);
      s_t0 = global_ns();
    }
    __syncthreads();
    const int pi = s_plant;
    const ServeMeta<T> M = meta[pi];
    const SolveBufs<T> B = ld_struct_cg(bufs + pi);   // written by the host at admission
    for (int k = threadIdx.x; k < M.nx; k += blockDim.x)
      M.x0s[k] = (T)(M.Sx[k] * *reinterpret_cast<const volatile double*>(&rq->x0[k]));
    if (!s_warm)
      for (long long e = threadIdx.x; e < M.nv; e += blockDim.x) B.V[e] = T(0);
    {
      int* c = reinterpret_cast<int*>(B.ctl);
      for (int k = threadIdx.x; k < (int)(sizeof(SolveCtl) / sizeof(int)); k += blockDim.x) c[k] = 0;
    }
    __threadfence();
    __syncthreads();
    batch_one<T, CH>(probs, B, tws, o, pi, g, smraw, s_prob, s_bar, s_ok, s_prof, first, nullptr);
    first = false;
    // result: u0 = u~0 / Su from T(v); the final iterate moved into V (warm start)
    const SolveCtl* c = B.ctl;
    const int fv = c->final_v & 3, ftv = c->final_tv & 3;
    T* bb[4] = {B.V, B.TV, B.VT, B.TVT};
    const T* z = bb[ftv];
    for (int k = threadIdx.x; k < M.nu; k += blockDim.x) rs->u0[k] = (double)ldc(z + M.o_u + k) / M.Su[k];
    if (threadIdx.x == 0) {
      rs->id = s_id;
      rs->status = c->status; rs->iters = c->iters; rs->n_T = c->n_T;
      rs->res_inf = c->res_inf;
      rs->risk = (double)ldc(z);
      rs->t_claim = s_t0;
      rs->t_done = global_ns();
    }
    __syncthreads();
    if (fv != 0)
      for (long long e = threadIdx.x; e < M.nv; e += blockDim.x) B.V[e] = ldc(bb[fv] + e);
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence_system();
      rs->done = 1;
      __threadfence_system();
      atomicMax(&dev->last_ns, (unsigned long long)global_ns());
      atomicSub(&dev->busy, 1);
    }
  }
}

template <class T, int CH>
cudaError_t launch_serve_ch(const Prob<T>* probs, const SolveBufs<T>* bufs, const int* tws, const ServeMeta<T>* meta,
                            const SolveOpts& o, const ServeReq* ring, ServeRes* res, int cap, ServeCtl* ctl,
                            ServeDev* dev, unsigned long long idle_ns, size_t smem, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_serve<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_serve<T, CH><<<grid, 256, smem, s>>>(probs, bufs, tws, meta, o, ring, res, cap, ctl, dev, idle_ns);
  return cudaGetLastError();
}

template <class T, int CH>
int serve_grid_ch(size_t smem, int* out) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaFuncSetAttribute(k_serve<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_serve<T, CH>, 256, smem) != cudaSuccess) return -1;
  *out = nsm * per;
  return 0;
}

template <class T, int CH>
cudaError_t launch_batch_ch(const Prob<T>* probs, const SolveBufs<T>* bufs, const int* tws, const SolveOpts& o,
                            const BatchPlan& plan, long long* cycles, size_t smem, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_batch<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const Prob<T>* a0 = probs;
  const SolveBufs<T>* a1 = bufs;
  const int* a2 = tws;
  SolveOpts a3 = o;
  BatchPlan a4 = plan;
  long long* a5 = cycles;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
  // cooperative: the gangs' barriers need their CTAs resident together
  return cudaLaunchCooperativeKernel((void*)k_batch<T, CH>, dim3(grid), dim3(256), args, smem, s);
}

template <class T, int CH>
int batch_grid_ch(size_t smem, int* out) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaFuncSetAttribute(k_batch<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<T, CH>, 256, smem) != cudaSuccess) return -1;
  *out = nsm * per;
  return 0;
}

template <class T, int CH>
cudaError_t launch_ch(const Prob<T>& P, const SolveBufs<T>& B, const SolveOpts& o, int tw,
                             int grid, int threads, cudaStream_t s) {
  const size_t smem = Views<T, CH>::bytes(threads, tw, P.pipe_bytes) + cta_smem_bytes(P);
  cudaError_t e = cudaFuncSetAttribute(k_solve<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  Prob<T> Pc = P;
  SolveBufs<T> Bc = B;
  SolveOpts oc = o;
  int twc = tw;
  void* args[] = {&Pc, &Bc, &oc, &twc};
  return cudaLaunchCooperativeKernel((void*)k_solve<T, CH>, dim3(grid), dim3(threads), args, smem, s);
}

template <class T, int CH>
int max_grid_ch(int tw, int threads, int pipe_bytes, size_t extra, int* out) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = Views<T, CH>::bytes(threads, tw, pipe_bytes) + extra;
  cudaFuncSetAttribute(k_solve<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve<T, CH>, threads, smem) != cudaSuccess)
    return -1;
  *out = nsm * per;
  return 0;
}

}  // namespace spock
