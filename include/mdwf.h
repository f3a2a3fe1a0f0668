/*
 * mdwf.h -- C ABI of libmdwf: the even-odd preconditioned Moebius domain-wall fermion
 * (MDWF) propagator solve of arXiv:1810.01609 on one NVIDIA GB300 (sm_103a).
 *
 * The paper (Sec. "Current State of the Art") states the problem this library solves:
 * linear solves of the domain-wall Dirac matrix on an L^3 x T x L5 x Nc x Ns space,
 * a radius-one stencil with small dense 12x12 diagonal blocks, by conjugate gradient
 * on the normal equations with red-black preconditioning, in "double-half" mixed
 * precision with reliable updates to double; the propagators feed Feynman-Hellmann
 * sequential solves and nucleon contractions (Sec. "Performance Measurement Method").
 *
 * Operator conventions (the paper prints none; these are the library's readings):
 *   chiral basis: gamma_k = [[0, i sigma_k], [-i sigma_k, 0]], gamma_4 = [[0,1],[1,0]],
 *   gamma_5 = diag(-1,-1,1,1), P_-/P_+ = upper/lower spin pair.
 *   H psi(x)  = sum_mu (1-gamma_mu) U_mu(x) psi(x+mu) + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)
 *   D_W       = (4 - M5) - H/2,  (B psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},
 *               psi_{Ls} -> -mf psi_0, psi_{-1} -> -mf psi_{Ls-1}
 *   D         = D_W (b5 + c5 B) + (1 - B)                 (Moebius 5D operator)
 *   D5 = b5 + c5 B,  A5 ("M5") = (4-M5) D5 + 1 - B
 *   M_pc      = 1 - (1/4) A5^-1 H_oe D5 A5^-1 H_eo D5        (odd sites; parity x+y+z+t)
 *
 * Layouts
 *   links   (user)  complex128 U[t][z][y][x][mu][a][b], mu = x,y,z,t; U_mu(x) lives on
 *                   the link x -> x+mu.  The time boundary phase t_bc is applied by the
 *                   library (do not fold it in).
 *   5D field (user) complex128 psi[rhs][s][t][z][y][x][spin][colour].
 *   4D field (user) complex128 psi[rhs][t][z][y][x][spin][colour].
 *   4D propagator   complex128 S[12][t][z][y][x][spin][colour]: column src_spin*3 +
 *                   src_colour holds the sink field of that source component (what
 *                   mdwf_project_4d writes for nrhs = 12 point sources).
 *   internal field  opaque device buffer of mdwf_field_bytes() bytes holding both
 *                   parities in the library's Ls-inner, site-blocked, 16-byte-chunk
 *                   layout for one precision and a given number of right-hand sides.
 *
 * Ownership: the caller owns every buffer passed in; the library never frees caller
 * memory.  The context owns its internal gauge copies, workspaces and tune cache.
 * Pointers flagged DEVICE must be device memory of the current CUDA device; pointers
 * flagged HOST are host memory (pinned is faster).  `stream` is a cudaStream_t (NULL =
 * legacy default stream).  All calls are stream-ordered; mdwf_solve* synchronise the
 * stream before returning so that `info` is valid.
 *
 * Errors: every int-returning call returns MDWF_SUCCESS (0) or a negative MDWF_ERR_*;
 * mdwf_strerror() names it.  Invalid arguments are rejected before any launch.
 */
#ifndef MDWF_H
#define MDWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum mdwf_status {
  MDWF_SUCCESS = 0,
  MDWF_ERR_ARG = -1,           /* invalid argument (null pointer, bad dims, Ls, op ...) */
  MDWF_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
  MDWF_ERR_OOM = -3,           /* device allocation failed */
  MDWF_ERR_NOT_SU3 = -4,       /* mdwf_load_gauge: a link is not special unitary */
  MDWF_ERR_NOT_CONVERGED = -5, /* maxiter reached; solution and info still written */
  MDWF_ERR_BREAKDOWN = -6,     /* CG breakdown: NaN/Inf or non-positive p^+ A p */
  MDWF_ERR_TIMEOUT = -7,       /* a bounded device-side wait gave up */
  MDWF_ERR_STATE = -8          /* call out of order (e.g. no gauge field loaded) */
};

enum mdwf_precision {
  MDWF_PREC_F64 = 0,   /* double storage, double arithmetic */
  MDWF_PREC_F32 = 1,   /* float storage, float arithmetic */
  MDWF_PREC_F16 = 2,   /* half storage + one float norm per 5D site, float arithmetic */
  MDWF_PREC_BF16 = 3,  /* bfloat16 storage, float arithmetic */
  MDWF_PREC_I16 = 4,   /* 16-bit fixed point (the paper's "16-bit fixed-point storage"): per
                          5D site one float norm = max |component| and 24 int16
                          q = RNE(32767 v / norm); links q = RNE(32767 u); float arithmetic
                          (CUDA-core hop only) */
  MDWF_PREC_F64E = 5   /* mdwf_apply / mdwf_field_bytes / mdwf_pack / mdwf_unpack only: FP64
                          storage (the MDWF_PREC_F64 layout) with the hops computed in
                          emulated FP64 -- every real split into a float pair hi + lo, SU(3)
                          products summed as compensated double-float sums (TwoSum, exact
                          FMA products), rounded to double once per output real: ~1e-14
                          relative, on the FP32 pipe; s-direction operators and epilogues in
                          FP64.  Not on a T-partitioned context (MDWF_ERR_STATE). */
};

enum mdwf_location { MDWF_HOST = 0, MDWF_DEVICE = 1 };

/* Operators of mdwf_apply.  "e"/"o" = even/odd half of the internal field; an op
 * writes only the half(s) it names and leaves the rest of `out` untouched. */
enum mdwf_op {
  MDWF_OP_HOP_EO = 0,      /* out_e = H_eo in_o                                   */
  MDWF_OP_HOP_OE = 1,      /* out_o = H_oe in_e                                   */
  MDWF_OP_HOP_EO_DAG = 2,  /* out_e = H_eo^+ in_o  (H^+ = gamma5 H gamma5)        */
  MDWF_OP_HOP_OE_DAG = 3,  /* out_o = H_oe^+ in_e                                 */
  MDWF_OP_D5 = 4,          /* out = (b5 + c5 B) in, both parities                 */
  MDWF_OP_D5_DAG = 5,
  MDWF_OP_M5 = 6,          /* out = A5 in, both parities                          */
  MDWF_OP_M5_DAG = 7,
  MDWF_OP_M5INV = 8,       /* out = A5^-1 in, both parities                       */
  MDWF_OP_M5INV_DAG = 9,
  MDWF_OP_HOP_EO_M5INV = 10, /* out_e = A5^-1 H_eo in_o : the fused hop + M5^-1 kernel */
  MDWF_OP_HOP_OE_M5INV = 11, /* out_o = A5^-1 H_oe in_e                            */
  MDWF_OP_MPC = 12,        /* out_o = M_pc in_o                                    */
  MDWF_OP_MPC_DAG = 13,    /* out_o = M_pc^+ in_o                                  */
  MDWF_OP_MDAGM = 14,      /* out_o = M_pc^+ M_pc in_o                             */
  MDWF_OP_FULL_D = 15,     /* out = D in (both parities)                           */
  MDWF_OP_FULL_D_DAG = 16, /* out = D^+ in                                         */
  MDWF_OP_MPC_SYM = 17,    /* out_o = M_sym in_o (symmetric form, see below)         */
  MDWF_OP_MPC_SYM_DAG = 18,/* out_o = M_sym^+ in_o                                 */
  MDWF_OP_COUNT = 19
};

/* Even-odd preconditioned forms of the odd-site system (mdwf_solve_params.pc_form).
 * The paper names red-black preconditioning without fixing the form.
 *   MDWF_PC_LEFT: M_pc = 1 - (1/4) A5^-1 H_oe D5 A5^-1 H_eo D5, solving M_pc x_o = b~_o.
 *   MDWF_PC_SYM:  the symmetric form of the rescaled operator D D5^-1, whose diagonal
 *                 block is A~ = A5 D5^-1:  M_sym = 1 - (1/4) A~^-1 H_oe A~^-1 H_eo with
 *                 A~^-1 = D5 A5^-1 (= D5 M_pc D5^-1), solving M_sym y = D5 b~_o and
 *                 x_o = D5^-1 y.  Its true residual is |D5 b~ - M_sym y| / |D5 b~|. */
enum mdwf_pc_form { MDWF_PC_LEFT = 0, MDWF_PC_SYM = 1 };

typedef struct mdwf_params {
  int dims[4];        /* X, Y, Z, T: each even and >= 2 */
  int Ls;             /* fifth-dimension extent, 2 <= Ls <= 32 */
  double b5, c5;      /* Moebius coefficients (b5 - c5 = 1 gives Shamir-like scaling) */
  double M5;          /* domain-wall height */
  double mf;          /* quark mass m_f */
  double t_bc;        /* time boundary phase (-1 antiperiodic, +1 periodic) */
  int gauge_recon;    /* 18: store all 18 reals of a link; 12: store two rows and
                         rebuild the third as conj(row0 x row1) */
  int check_su3;      /* nonzero: mdwf_load_gauge rejects links with |U U^+ - 1| or
                         |det U - 1| above 1e-9 (MDWF_ERR_NOT_SU3) */
  int t_ranks;        /* T partitions of the global lattice (1: the context holds it all) */
  int t_rank;         /* this context's partition: global timeslices
                         [t_rank * dims[3], (t_rank + 1) * dims[3]); dims[3] is the LOCAL
                         extent (even), the global one is t_ranks * dims[3] */
  int f64_emulation;  /* nonzero (default): the FP64 hops of a mixed-precision solve --
                         preparing b~, the reliable-update anchors before the convergence
                         check, reconstructing x_e -- and of mdwf_make_source_4d run in
                         emulated FP64 (see MDWF_PREC_F64E); a solve's convergence is always
                         decided on a residual computed in native FP64, and a plain FP64
                         solve (sloppy_prec MDWF_PREC_F64) is native FP64 throughout.
                         Ignored on a T-partitioned context. */
} mdwf_params;

typedef struct mdwf_solve_params {
  double tol;          /* target true relative residual |b~ - M_pc x| / |b~| */
  int maxiter;         /* inner iteration cap */
  int sloppy_prec;     /* MDWF_PREC_F64: plain FP64 CG; F32/F16/BF16: mixed-precision CG
                          whose inner iterations store fields in that precision and
                          reliable-update to FP64 */
  double delta;        /* reliable update when |r| < delta * max |r| since the last one */
  int ru_interval;     /* ... or after this many inner iterations */
  int check_interval;  /* iterations between host polls (and per captured CUDA graph) */
  int use_graph;       /* nonzero: replay the check_interval iterations as a CUDA graph */
  int location;        /* MDWF_HOST or MDWF_DEVICE for src / sol */
  int full_residual;   /* nonzero: also compute |b - D x| / |b| (a diagnostic: two extra
                          FP64 hops and a full-lattice FP64 pass) */
  int pc_form;         /* MDWF_PC_LEFT or MDWF_PC_SYM */
} mdwf_solve_params;

typedef struct mdwf_solve_info {
  int status;              /* MDWF_SUCCESS or MDWF_ERR_NOT_CONVERGED / _BREAKDOWN */
  int iterations;          /* inner CG iterations */
  int reliable_updates;    /* reliable updates (mixed precision): x64 += x_s and the inner
                              residual restarted from res = b~ - M x64 */
  double true_residual;    /* FP64 relative residual of the odd-site system solved: LEFT
                              |b~ - M_pc x_o| / |b~|, SYM |D5 b~ - M_sym y| / |D5 b~| */
  double full_residual;    /* FP64 |b - D x| / |b| (if requested, else -1) */
  double time_ms;          /* wall time of the call (host clock, stream synchronised) */
  int fp64_residuals;      /* residuals b~ - M_pc x recomputed with M_pc in FP64 (the others
                              are updated as res -= M_pc x_s with M_pc in FP32) */
  int emulated_residuals;  /* of those, how many ran in emulated FP64 (f64_emulation) */
} mdwf_solve_info;

typedef struct mdwf_ctx mdwf_ctx;

/* Fill *p with defaults: dims 4^4, Ls 8, b5 1.5, c5 0.5, M5 1.3, mf 0.05, t_bc -1,
 * recon 18, check_su3 1, t_ranks 1, t_rank 0, f64_emulation 1. */
void mdwf_default_params(mdwf_params* p);
/* Defaults: tol 1e-10, maxiter 100000, sloppy F16, delta 0.05, ru_interval 100,
 * check_interval 10, use_graph 1, location DEVICE, full_residual 0, pc_form LEFT. */
void mdwf_default_solve_params(mdwf_solve_params* sp);

/* Create a context on the current CUDA device.  Validates the parameters
 * (MDWF_ERR_ARG).  Allocates nothing on the device until a gauge field is loaded. */
int mdwf_create(const mdwf_params* p, mdwf_ctx** out);
/* Free every device buffer of the context and the context itself (NULL is a no-op). */
void mdwf_destroy(mdwf_ctx* ctx);

/* Load the gauge links (user layout above, complex128; `where` = MDWF_HOST/DEVICE) into
 * the context's internal SoA layout: per parity and site, the 4 forward links U_mu(x) and
 * the 4 backward links U_mu(x-mu)^+ with the boundary phase folded in.  The lower
 * precision copies are made on first use.  Returns MDWF_ERR_NOT_SU3 if check_su3 is set
 * and a link is not in SU(3).  A T-partitioned context (t_ranks > 1) takes dims[3] + 1
 * timeslices: first the last timeslice of the partition below (global timeslice
 * t_rank * dims[3] - 1, periodically; only its t links are read), then its own. */
int mdwf_load_gauge(mdwf_ctx* ctx, const double* links, int where, void* stream);

/* Bytes of one internal field (both parities) of precision `prec` and nrhs right-hand
 * sides. */
int mdwf_field_bytes(const mdwf_ctx* ctx, int prec, int nrhs, size_t* bytes);

/* user5d (DEVICE, complex128 [nrhs][s][t][z][y][x][4][3]) -> internal field (DEVICE).
 * F16 stores per 5D site norm = float(max |component|) and halves = RNE(v / norm); I16
 * the same norm and int16 RNE(32767 v / norm) (FP64 product, then quotient); BF16 and
 * F32 are RNE conversions. */
int mdwf_pack(mdwf_ctx* ctx, const double* user5d, void* internal, int prec, int nrhs,
              void* stream);
/* internal field (DEVICE) -> user5d (DEVICE, complex128). */
int mdwf_unpack(mdwf_ctx* ctx, const void* internal, double* user5d, int prec, int nrhs,
                void* stream);

/* out = op(in) on internal fields (DEVICE, precision prec, nrhs right-hand sides).
 * `in` and `out` must not overlap.  Needs a loaded gauge field (MDWF_ERR_STATE). */
int mdwf_apply(mdwf_ctx* ctx, int op, int prec, const void* in, void* out, int nrhs,
               void* stream);

/* Solve D x = b for one 5D source: b~_o = A5^-1 (b_o + H_oe D5 A5^-1 b_e / 2), CG on
 * M_pc^+ M_pc to |b~ - M_pc x_o| <= tol |b~| (FP64-recomputed), then
 * x_e = A5^-1 (b_e + H_eo D5 x_o / 2).  src/sol are user 5D fields at sp->location.
 * Returns MDWF_SUCCESS, MDWF_ERR_NOT_CONVERGED (solution still written) or an error.
 * With env MDWF_VERBOSE=1 every reliable update / residual check prints one line on
 * stderr (iteration, kind: FP64 recomputation or FP32 incremental update, residual);
 * MDWF_VERBOSE=2 also recomputes the FP64 residual at incremental updates (diagnostic). */
int mdwf_solve(mdwf_ctx* ctx, const double* src, double* sol,
               const mdwf_solve_params* sp, mdwf_solve_info* info, void* stream);
/* The same for nrhs sources in one batched solve (contiguous [nrhs][...] user fields);
 * link loads are shared across the right-hand sides and each has its own CG scalars.
 * info points to nrhs entries.  The return value is the worst status. */
int mdwf_solve_multi(mdwf_ctx* ctx, int nrhs, const double* src, double* sol,
                     const mdwf_solve_params* sp, mdwf_solve_info* info, void* stream);

/* 4D source -> 5D source: eta = D(mf=1) P (b at s=0), (P psi)_s = P_- psi_s + P_+ psi_{s+1}
 * (Pauli-Villars injection; q below is then D_eff^-1 b).  src4d [nrhs][t][z][y][x][4][3],
 * src5d [nrhs][s][...], both complex128 at `where`. */
int mdwf_make_source_4d(mdwf_ctx* ctx, const double* src4d, double* src5d, int nrhs,
                        int where, void* stream);
/* 5D solution -> 4D propagator column q = P_- y_0 + P_+ y_{Ls-1}. */
int mdwf_project_4d(mdwf_ctx* ctx, const double* sol5d, double* q4d, int nrhs, int where,
                    void* stream);
/* Propagator columns in one call (Sec. "Performance Measurement Method": the propagator
 * solve from a 4D source): q = P_- y_0 + P_+ y_{Ls-1} with D y = D(mf=1) P (b at s=0),
 * i.e. mdwf_make_source_4d, mdwf_solve_multi and mdwf_project_4d chained on the device.
 * src4d and q4d are [nrhs][t][z][y][x][4][3] complex128 at `where` (MDWF_HOST or
 * MDWF_DEVICE); the 5D source and solution stay in one device workspace of the context
 * (nrhs * Ls * 4D-field bytes), so a host caller moves only the 4D fields.  sp is used as
 * for mdwf_solve_multi except sp->location (ignored).  info points to nrhs entries.
 * Returns the solve's worst status (MDWF_ERR_NOT_CONVERGED: q still written) or an error. */
int mdwf_propagator(mdwf_ctx* ctx, int nrhs, const double* src4d, double* q4d, int where,
                    const mdwf_solve_params* sp, mdwf_solve_info* info, void* stream);
/* Feynman-Hellmann sequential source (Sec. "Current State of the Art": all temporal
 * distances for the cost of one): out(z) = gamma_3 gamma_5 q(z) at every site z of every
 * timeslice, for nrhs 4D columns. */
int mdwf_fh_source(mdwf_ctx* ctx, const double* q4d, double* out4d, int nrhs, int where,
                   void* stream);
/* Nucleon two-point function C(t) = sum_x Tr[(1+gamma_4)/2 G(x)] of
 * N = eps_abc (u_a^T C gamma_5 d_b) u_c, C = gamma_2 gamma_4, with both Wick terms of the
 * two u lines (u1 = line of the sink u_a, u2 = line of the sink u_c) and the d line, in
 * FP64.  u1, d, u2 are 4D propagators (12-column layout above); corr receives T complex values
 * (2T doubles).  All at `where`. */
int mdwf_contract_nucleon(mdwf_ctx* ctx, const double* u1, const double* d,
                          const double* u2, double* corr, int where, void* stream);

/* Feynman-Hellmann effective coupling (Sec. "Current State of the Art": one sequential
 * solve with the current at every time gives all source-sink separations): with
 * R(t) = Re[C_FH(t) / C(t)], geff[t] = R(t+1) - R(t) for t = 0 .. T-2, whose large-t value
 * is the matrix element (g_A for the gamma_3 gamma_5 current).  c2 = C(t) and c3 = C_FH(t)
 * are T complex values (2T doubles, HOST), e.g. mdwf_contract_nucleon of S,S,S and the sum
 * of the contractions with the FH propagator on either u line; geff receives T - 1
 * doubles (HOST).  MDWF_ERR_ARG if T < 2 or some C(t) is zero or not finite. */
int mdwf_fh_effective_coupling(const double* c2, const double* c3, double* geff, int T);

/* Allocation-free nucleon contraction (the paper has no counterpart; it serves callers
 * that cannot allocate device memory: code running during CUDA graph capture, programs
 * whose device memory belongs to a pool allocator that forbids other allocations, hosts
 * that plan every byte of device memory up front).  Computes exactly what
 * mdwf_contract_nucleon computes, for DEVICE pointers only (u1, d, u2: 12-column 4D
 * propagators; corr: T complex values), without any cudaMalloc or cudaFree: the per-site
 * scratch lives in a fixed 8 MiB array inside the library, which every GPU that loads the
 * library keeps until the process exits.  Lattices with more than 524288 4D sites are
 * rejected with MDWF_ERR_ARG (use mdwf_contract_nucleon), and so is a context created on
 * another device than the current one.  Outside stream capture every call looks up the
 * array's device address on the current device; a call made while `stream` is being
 * captured reuses the address of this device's last uncaptured call, so make one call on
 * each device before any capture (MDWF_ERR_STATE otherwise).  All calls share the array:
 * calls whose kernels overlap on the GPU (different streams, or the same call issued from
 * several threads) race and must be serialised by the caller.  Detail of a failure:
 * mdwf_noalloc_last_error(). */
int mdwf_contract_nucleon_noalloc(const mdwf_ctx* ctx, const double* u1, const double* d,
                                  const double* u2, double* corr, void* stream);
const char* mdwf_noalloc_last_error(void);

/* Autotuner control: enable (1) / disable (0) brute-force launch tuning (default from
 * env MDWF_TUNE, on).  The cache is a std::map keyed by kernel, lattice, Ls, nrhs,
 * precision and mode; MDWF_TUNE_CACHE names a JSON file it is loaded from and saved to. */
int mdwf_set_tuning(mdwf_ctx* ctx, int enable);
/* Number of tune-cache entries, and the tuned sites-per-CTA of entry i with its time (ms)
 * and key (copied into key[keylen]).  For the fused 32-bit hop kernels the tuner also
 * chooses between two builds: 65536 is added to sites_per_cta when it picked the
 * occupancy-bounded one (at most 64 registers per thread). */
int mdwf_tune_entries(const mdwf_ctx* ctx, int* count);
int mdwf_tune_entry(const mdwf_ctx* ctx, int i, char* key, int keylen, int* sites_per_cta,
                    double* ms);

/* Number of kernels this context has launched so far (all streams). */
long long mdwf_launch_count(const mdwf_ctx* ctx);
/* Algorithmic HBM bytes of every kernel this context has launched so far: each field a
 * kernel reads or writes counted once per 5D site (F64 192 B, F32 96 B, F16 48 B + 4 B
 * norm, BF16 48 B), links once per launch (8 per output 4D site, 18 or 12 reals), user
 * complex128 fields at 192 B per 5D site. */
double mdwf_algorithmic_bytes(const mdwf_ctx* ctx);

/* ---------------------------------------------------------------- T-partitioned lattice
 * (Sec. "Current State of the Art": the radius-one stencil is decomposed across GPUs,
 * faces are exchanged and the interior is computed while they travel.)  A context with
 * t_ranks > 1 holds dims[3] timeslices of the global lattice.  Every hop it applies packs
 * the two faces of its input half -- per site of its first and of its last timeslice
 * and per column, the 12 reals of the half spinor (1 -/+ sig gamma_4) psi the receiving
 * hop needs, in the compute type (double for F64, float otherwise), followed for F16 and
 * int16 by one float scale per site and column -- launches the interior timeslices, calls the face
 * exchange, then launches the first and last timeslices, which take their t neighbours
 * across the boundary from the received faces.  The result is bit-identical to the
 * undecomposed operator's.  Operators whose kernels reduce over the lattice (the CG
 * iteration) need a global sum and are not available: mdwf_solve* return MDWF_ERR_STATE.
 *
 * The exchange moves `bytes` bytes: send_lo (faces of this partition's first timeslice)
 * to the partition below, which receives it as its recv_hi; send_hi (last timeslice) to
 * the partition above, received as recv_lo; periodic in t_rank.  It must have completed
 * the transfers in the order of `stream` when it returns 0 (nonzero: an error status
 * that the calling apply returns). */
typedef int (*mdwf_face_exchange_fn)(void* user, const void* send_lo, const void* send_hi, void* recv_lo,
                                     void* recv_hi, size_t bytes, void* stream);
/* Set the face exchange of a partitioned context (fn NULL: none). */
int mdwf_set_face_exchange(mdwf_ctx* ctx, mdwf_face_exchange_fn fn, void* user);
/* Bytes of one face of precision prec and nrhs right-hand sides. */
int mdwf_face_bytes(const mdwf_ctx* ctx, int prec, int nrhs, size_t* bytes);
/* Use caller-owned device buffers (each at least mdwf_face_bytes for the precisions and
 * right-hand sides applied) for the faces instead of the context's own; NULLs: back to
 * the context's own. */
int mdwf_set_face_buffers(mdwf_ctx* ctx, void* send_lo, void* send_hi, void* recv_lo, void* recv_hi,
                          size_t bytes);
/* Exchange faces among the n partitions of one lattice held by contexts of this process
 * (ctxs[k] has t_rank k): sets each context's exchange to an in-process one that copies
 * the neighbours' send faces into its receive buffers.  Each context must then be driven
 * by its own host thread (one stream each), all applying the same operator at once: the
 * exchange waits for the other partitions at a host barrier and gives up with
 * MDWF_ERR_TIMEOUT after 60 s.  The group lives until its last context is destroyed. */
int mdwf_group_partitions(mdwf_ctx* const* ctxs, int n);

/* Name of a status code. */
const char* mdwf_strerror(int status);
/* Detail of the last failure on the calling host thread (empty if none). */
const char* mdwf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MDWF_H */
