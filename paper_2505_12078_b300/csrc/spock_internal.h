// spock_internal.h -- host-side declarations shared by the .cu files of libspock.
#pragma once
#include <cuda_runtime.h>

#include "spock_dev.cuh"

namespace spock {

// Pointers and sizes of the offline (FP64) setup.
struct SetupArgs {
  int n, n_nl, nx, nu, nbx, nbu, has_ball;
  int ldB, ldF, ldP, ldK;
  double a_con, a_conN;
  const int* anc;
  const int* ch_off;
  const double* prob;
  const double *Sx, *SxN, *Su;
  // raw data
  const double *A, *B, *c, *Qd, *Rd, *QNd, *xlo, *xhi, *ulo, *uhi, *uball;
  // scaled dynamics
  double *At, *Bt, *ct;
  // Alg. 1
  double *P, *K, *Rt, *Lc, *Linv, *Rinv, *KA, *BtP, *PAb, *Abar;
  int* err;
  // iteration data (FP64)
  double *MB, *MF, *MP, *KT, *Pc, *kc;
  double *qh, *rh, *qNh, *gx, *gu, *gN, *box_lo, *box_hi, *boxN_lo, *boxN_hi, *ball;
  int ys_block = 1;         // the closed form of AV@R's (y, s) blocks (0: computed on the host)
  const double* soft_w = nullptr;   // soft costs: 1/s per component of (x, u), or null
  double xu_shift = 0.0;   // added to every diagonal entry of the (x^i, u^i) blocks of L'L (l1 rows)
};

cudaError_t launch_scale_dyn(const SetupArgs& a, cudaStream_t s);
cudaError_t launch_alg1(const SetupArgs& a, const int* stage_off_host, int N, cudaStream_t s);
cudaError_t launch_build(const SetupArgs& a, cudaStream_t s);
cudaError_t launch_norm_L(const SetupArgs& a, unsigned long long* out, cudaStream_t s);
cudaError_t launch_convert_f64_f32(const double* a, float* b, long long n, cudaStream_t s);
// nmat matrices rows x cols (leading dim lds) -> output-column-major, each
// column padded to ldd rows with zeros; dst is double (prec 64) or float (32)
cudaError_t launch_transpose(const double* src, long long nmat, int rows, int cols, int lds, int ldd,
                             void* dst, int prec, cudaStream_t s);
cudaError_t launch_convert_f32_f64(const float* a, double* b, long long n, cudaStream_t s);

template <class T>
cudaError_t launch_apply_L(const Prob<T>& P, const int* ynode, const T* z, T* eta, cudaStream_t s);
// centred FP32 iteration (spock_centre.cu): the centre's data from T(c) and
// L z_c, the move of an increment into the centre, an FP32 copy of it
cudaError_t launch_centre(const Prob<double>& P, const double* c, const double* tc, const double* lz, double alpha,
                          float* cz, double* A, double* B, cudaStream_t st);
cudaError_t launch_centre_move(long long n, double* c, const float* d, cudaStream_t st);
cudaError_t launch_centre_to_f32(long long n, const double* c, float* v, cudaStream_t st);
template <class T>
cudaError_t launch_apply_Lt(const Prob<T>& P, const int* ynode, const T* eta, T* z, cudaStream_t s);

// full weights, linear terms, ||L|| with full blocks (spock_setup_ext.cu)
cudaError_t launch_chol_upper(int nmat, int m, double* W, int* err, cudaStream_t s);
cudaError_t launch_ftinv(int nblk, int m, int full, const double* F, const double* lin, double* w, double* kap,
                         cudaStream_t s);
cudaError_t launch_translation(int nblk, int mx, int mu, const double* wx, const double* wu, const double* kap,
                               double* a, cudaStream_t s);
cudaError_t launch_scale_factor(long long nblk, int m, const double* F, const double* S, double* Ft, double* FtT,
                                cudaStream_t s);
cudaError_t launch_norm_L_blocks(const Prob<double>& P, unsigned long long* out, cudaStream_t s);

// FP64 exit check (Sec. 5.3): xi1, xi2, primal infeasibility, complementarity
// gap of (v, T(v)); see spock_diag.cu for the scratch it needs
size_t diag_partials_doubles();
cudaError_t launch_diagnostics(const Prob<double>& P, const int* ynode, const double* v, const double* tv,
                               double* d, double* ltde, double* ldz, double* lz, double* part, double* out6,
                               cudaStream_t s);

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------
struct SolveOpts {
  double tol;
  int max_iters;
  int max_backtracks;
  int method;          // 0 SPOCK, 1 plain CP, 2 one T evaluation
  double rank_tol;     // Anderson rank test (relative to ||Y||_F)
  unsigned long long wait_ns;   // limit of one grid-barrier wait (0: BARRIER_LIMIT_NS)
  int phantom;         // test hook: CTAs a single-problem launch's barriers expect beyond its grid
  int aa_qr;           // 1: Anderson least squares by an updated QR factorisation (Y slots hold Q)
};

// Device control block of one solve (global memory, zeroed before a launch).
struct SolveCtl {
  GridCtl bar;
  int status;          // 0 ok, 1 maxiter, <0 error
  int iters, n_T, n_K0, n_K1, n_K2, n_fb, n_bt;
  double res_inf;
  double zeta, omega_safe;
  double red[NRED];    // result of the last group reduction
  double stats[NRED];  // reduction of the last T evaluation of the final iterate
  int final_v;         // index (0..3 of V, TV, VT, TVT) holding the final iterate v
  int final_tv;        // index holding T(v)
  int diag[4];         // first bulk-copy wait that gave up: CTA, barrier, parity, site
  int check_site;      // bounds-checked build: the first index check that failed (0: none)
  // device time per phase seen by CTA 0 (ns, barrier waits included):
  // 0 prep, 1 backward sweep, 2 forward sweep, 3 T reduction, 4 Anderson dots,
  // 5 direction pass, 6 K2/backtrack passes, 7 count of T evaluations;
  // 8.. SM cycles seen by thread 0 of CTA 0 inside the backward sweep:
  // 8 bulk-copy waits, 9 mat-vecs, 10 team reductions, 11 steps, 12 grid
  // barriers, 13 all-reductions, 14 barrier count, 15 all-reduce count
  unsigned long long prof[16];
};

template <class T>
struct SolveBufs {
  T *V, *TV, *VT, *TVT, *PSI, *VP, *RP;   // n_v each
  T *S, *Y;                               // 3 slots of sstride each
  long long sstride;                      // n_v rounded up to a multiple of 4
  double* partials;                        // [2][grid][NRED]
  unsigned* flags;                         // [grid] barrier flags
  SolveCtl* ctl;
};

// Schedule of the batched launch: gangs of CTAs for large problems, single
// CTAs for the rest (see k_batch).
struct BatchPlan {
  int n_gang_ctas;          // CTAs 0 .. n_gang_ctas-1 belong to gangs
  const int* gang_of;       // [n_gang_ctas] gang of the CTA
  const int* gang_start;    // [gangs] first CTA of the gang
  const int* gang_size;     // [gangs]
  const int* list_off;      // [gangs + 1] into list
  const int* list;          // problems of every gang, in order
  unsigned* flags;          // barrier flags: CTA c uses flags[c] (zeroed before the launch)
  double* partials;         // 2 x n_gang_ctas x NRED per gang, at 2 NRED gang_start
  const int* small_order;   // problems solved by single CTAs, largest first
  int n_small;
  int* next;                // queue position of small_order (zeroed before the launch)
};

// Serving: requests and results live in mapped host memory. The host fills a
// request slot, then publishes it by raising `tail`; a CTA of the persistent
// k_serve claims it, solves the plant's problem from the request's x0 (warm
// from the plant's resident iterate if asked), writes the result slot and
// raises its `done` word.
constexpr int SERVE_MAX_NX = 64;
constexpr int SERVE_MAX_NU = 64;
struct ServeReq {
  int plant;             // index into the server's plants
  int warm;              // 1: start from the plant's last iterate
  long long id;          // request id (echoed)
  double x0[SERVE_MAX_NX];
};
struct ServeRes {
  long long id;
  int status, iters, n_T, pad;
  double res_inf, risk;
  double u0[SERVE_MAX_NU];   // the first control, unscaled
  unsigned long long t_claim, t_done;   // device global timer (ns)
  volatile int done;         // raised last (release), cleared by the host
  int pad2;
};
struct ServeCtl {
  volatile long long tail;   // requests published by the host
  volatile int stop;         // host: leave now
  int pad;
};
struct ServeDev {             // device-side state of the serving launch
  long long head;              // requests claimed
  unsigned long long last_ns;  // global timer at the last claim or completion
  int busy;                    // CTAs solving a request
  int pad;
};
template <class T>
struct ServeMeta {           // per plant: what a request needs beyond Prob / SolveBufs
  int nx, nu;
  long long o_u, nv;
  const double* Sx;
  const double* Su;
  T* x0s;
};

template <class T>
cudaError_t launch_solve(const Prob<T>& P, const SolveBufs<T>& B, const SolveOpts& o, int tw,
                         int grid, int threads, cudaStream_t s);
int solver_max_grid(int precision, int tw, int threads, int D, int pipe_bytes, size_t extra, int* grid_out);
size_t solver_smem_bytes(int precision, int tw, int threads, int D, int pipe_bytes);
int solver_chunks(int precision, int width);

}  // namespace spock

struct spock_problem;
namespace spock {
int op_T_with_scratch(spock_problem* p, int precision, const void* v_in, void* v_out,
                      double* stats, cudaStream_t st, unsigned char* scratch, size_t bytes);
}  // namespace spock
