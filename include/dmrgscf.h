/*
 * dmrgscf.h -- C-ABI of the GB300 spin-adapted DMRG / CAS-SCF hot path.
 *
 * Method: arXiv:2503.20700, "Orbital optimization of large active spaces via
 * AI-accelerators".  The library implements the DMRG-CI side of the paper's
 * DMRG-SCF: the spin-adapted (SU(2) x U(1)) two-site DMRG sweep of Sec. II.B-D
 * (Davidson with the effective-Hamiltonian product H_eff psi, decimation to
 * D SU(2) multiplets, operator renormalisation), the one- and two-particle
 * RDMs of Eqs. onerdm/twordm/rdm1_su2, and the integral transformation and
 * orbital gradient of the CAS-SCF step of Sec. II.A.
 *
 * Conventions shared by all entry points
 *  - All array arguments are HOST pointers to row-major float64 data unless
 *    stated otherwise; the library copies inputs and writes caller-allocated
 *    outputs.  The caller keeps ownership of every pointer.
 *  - Integrals are in chemists' notation: eri[((p*n+q)*n+r)*n+s] = (pq|rs),
 *    the Hamiltonian of Sec. II.A being
 *        H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps).
 *  - Spin quantum numbers are passed doubled (two_s = 2S).
 *  - Every call returns a dmrg_status; the library never aborts or exits.
 *    On error the message is available from dmrg_last_error().
 *  - All floating-point work runs on the CUDA device (sm_103a).  There is no
 *    host fallback: without a usable GPU the calls return DMRG_ECUDA.
 */
#ifndef DMRGSCF_H
#define DMRGSCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmrg_ctx dmrg_ctx;

typedef enum {
  DMRG_OK = 0,
  DMRG_EINVAL = -1,    /* bad argument (sizes, parity, NULL pointer)        */
  DMRG_ENOMEM = -2,    /* device allocation failed                           */
  DMRG_ECUDA = -3,     /* CUDA error or no usable device                     */
  DMRG_ENOCONV = -4,   /* Davidson did not reach the tolerance               */
  DMRG_ETIMEOUT = -5,  /* a bounded device wait ran out                      */
  DMRG_ESTATE = -6,    /* call out of order (e.g. RDMs before any sweep)     */
  DMRG_EINTERNAL = -7  /* internal inconsistency (reported, never aborted)   */
} dmrg_status;

typedef enum {
  DMRG_FP64 = 0,        /* all GEMMs in float64                              */
  DMRG_SPLIT_TF32 = 1,  /* H_eff psi / renormalisation GEMMs as 3xTF32 with
                           FP32 accumulation; Davidson, eigensolver and the
                           final reductions stay float64                      */
  DMRG_BF16X9 = 2,      /* reserved: BF16x9 split products (not available)   */
  DMRG_SPLIT_HPSI = 3,  /* 3xTF32 in the H_eff psi GEMMs only; renormalisation
                           and complementary-operator GEMMs in float64          */
  DMRG_SPLIT_HPSI_TC = 4, /* as DMRG_SPLIT_HPSI, with the H_eff psi split products
                           issued on the tcgen05 tensor cores (TMEM
                           accumulators, 128 x 256 sigma tiles, operands
                           pre-split into TF32 hi/lo planes); a bounded wait
                           that runs out returns DMRG_ETIMEOUT              */
  DMRG_SPLIT_ALL_TC = 5  /* as DMRG_SPLIT_HPSI_TC, with the renormalisation
                           O' = U^T O U (Sec. II.B) also one tcgen05
                           contraction per group of operators (operator
                           blocks and U as TF32 plane pairs, float-pair
                           partial sums); complementary-operator GEMMs stay
                           float64                                           */
} dmrg_precision;

typedef struct {
  int D;                  /* bond dimension in SU(2) multiplets (Sec. II.C)  */
  int max_davidson_iter;  /* per bond                                        */
  double davidson_tol;    /* ||H_eff psi - E psi|| with ||psi|| = 1 (Sec. II.D) */
  int precision;          /* dmrg_precision                                  */
  int max_space;          /* Davidson subspace size before restart           */
  int verbose;            /* 0 quiet, 1 per bond, 2 per Davidson step        */
  int device;             /* CUDA device ordinal                             */
  int strict_convergence; /* 1: dmrg_sweep / dmrg_sweep_part return
                             DMRG_ENOCONV (after completing the sweep, state
                             intact) when a bond's Davidson stopped at
                             max_davidson_iter above davidson_tol             */
  int debug_bounds;       /* 1: every tcgen05 task list is checked on the host
                             against its pool, scratch and item ranges before
                             its first launch (DMRG_EINTERNAL on a violation) */
  uint64_t seed;          /* seed of the Davidson start vector where no
                             predicted wavefunction exists (0: fixed default) */
  size_t hbm_budget_bytes;/* 0: no cap.  Otherwise the device memory the
                             context may hold: an allocation beyond it fails
                             with DMRG_ENOMEM unless stored blocks can be moved
                             to pinned host memory (see dmrg_sweep)            */
  double wait_timeout_s;  /* bound of every device-side wait (default 2 s; 0:
                             a wait not complete at its first probe gives up)
                             -- a wait that runs out returns DMRG_ETIMEOUT     */
  double trunc_target;    /* 0: keep D multiplets at every bond.  > 0: dynamic
                             bond dimension (Sec. II.D): keep the fewest
                             multiplets whose discarded weight is at most
                             trunc_target, between D_min and D                */
  int D_min;              /* lower bound of the dynamic bond dimension        */
  int rq64_every_bond;    /* 1: with a split precision, every bond energy (not
                             only the sweep energy) is the float64 Rayleigh
                             quotient of its eigenvector (one float64 H_eff psi
                             per bond)                                        */
  int tc_drain_terms;     /* DMRG_SPLIT_HPSI_TC: FP32 accumulation length of the
                             tcgen05 contraction's sigma tile between drains
                             into its float-pair partial tile, in terms of
                             psi's column index (sum of kb over items; 0:
                             after every item; default 1024) -- shorter is
                             slightly more accurate and slower                */
  int tc_autotune;        /* 1: DMRG_SPLIT_HPSI_TC / DMRG_SPLIT_ALL_TC pick the
                             schedule of each H_eff psi launch (tile width,
                             item chunks per CTA, task order; see
                             dmrg_tc_shape_candidates) by timing: the first
                             products with a new sector histogram run the
                             candidate schedules in turn (every one computes
                             the full product) and the fastest is kept for
                             that histogram.  0 (default): the first candidate.
                             Results differ between schedules only by FP32
                             summation order                                  */
} dmrg_opts;

/* Fill *o with defaults: D=64, 200 iterations, tol 1e-10, FP64, space 24,
 * no budget, wait bound 2 s, fixed D (trunc_target 0, D_min 1). */
void dmrg_default_opts(dmrg_opts* o);

/*
 * dmrg_init -- set up the DMRG-CI problem of one active space.
 *   n         number of active orbitals (sites), n >= 2
 *   h         n*n one-electron integrals (symmetric)
 *   eri       n^4 two-electron integrals (pq|rs), or NULL if chol is given
 *   chol      rank*n*n Cholesky vectors L^k_pq with (pq|rs) = sum_k L^k_pq L^k_rs,
 *             or NULL if eri is given
 *   e_core    constant energy added to every reported energy
 *   n_elec    number of active electrons N (0..2n)
 *   two_s     2S of the target multiplet (parity of n_elec)
 *   opts      options, or NULL for the defaults
 *   occ       optional n site occupations (0/1/2) of the initial product state
 *   two_s_right optional n+1 doubled spins of the right blocks of that state
 *             (sites i..n-1, coupled from the right); both NULL for the
 *             default state (electrons spread evenly, minimal spins)
 * The initial right blocks are built on the device before returning.
 * Returns DMRG_EINVAL for inconsistent sizes/parities, DMRG_ECUDA without a
 * device, DMRG_ENOMEM if the device memory is exhausted.
 */
dmrg_status dmrg_init(dmrg_ctx** out, const double* h, const double* eri, const double* chol,
                      int rank, double e_core, int n, int n_elec, int two_s, const dmrg_opts* opts,
                      const int* occ, const int* two_s_right);

/*
 * dmrg_sweep -- run n_sweeps full sweeps (L->R over bonds 0..n-3, then R->L
 * over bonds n-2..1; Sec. II.B two-site DMRG).  *energy receives the Davidson
 * eigenvalue of the last bond plus e_core, *max_trunc_err the largest
 * discarded weight of the last sweep.  Either output may be NULL.  With a
 * split precision the reported energy is the float64 Rayleigh quotient of
 * the last bond's eigenvector (one float64 H_eff psi).
 *
 * Device memory: besides the stored blocks of every bond, the context keeps
 * each bond's enlarged block (block plus site) for the opposite half-sweep,
 * which needs it again.  A block is kept only while the context holds at most 40%
 * of the device's memory and at least 20% of it is still free.  Kept blocks
 * are released by dmrg_set_precision, dmrg_rdm12 and dmrg_free.
 */
dmrg_status dmrg_sweep(dmrg_ctx* ctx, int n_sweeps, double* energy, double* max_trunc_err);

/*
 * dmrg_sweep_part -- part of a sweep (Sec. II.B two-site DMRG): direction 0
 * runs L->R over bonds 0..last_bond (starting a sweep), direction 1 runs
 * R->L over bonds n-2..last_bond (after a completed L->R half-sweep).
 * Afterwards the context holds the blocks of the next bond in that
 * direction (last_bond+1, or last_bond-1), where dmrg_bond_solve can run.
 * Outputs as for dmrg_sweep (energy of bond last_bond).  DMRG_EINVAL for a
 * bond out of range, DMRG_ESTATE for an R->L part without its left blocks.
 * dmrg_rdm12 needs a sweep that ended at bond 1 (a full sweep).
 */
dmrg_status dmrg_sweep_part(dmrg_ctx* ctx, int direction, int last_bond, double* energy,
                            double* max_trunc_err);

/* Result of dmrg_bond_solve (energies include e_core). */
typedef struct {
  double energy;          /* Davidson eigenvalue in the product's precision   */
  double energy_rq64;     /* float64 Rayleigh quotient of the returned vector */
  double residual64;      /* float64 ||H_eff psi - E_rq psi||, ||psi|| = 1    */
  double gap;             /* second minus lowest Ritz value at exit           */
  int iterations;         /* Davidson iterations                              */
  int calls;              /* H_eff psi products (timed)                       */
  double flops_per_call;  /* algorithmic FLOPs of one product (2mnk, once)    */
  double ms_total;        /* CUDA-event milliseconds of all products          */
  int64_t dim;            /* length of the two-site wavefunction              */
  double contraction_ms;  /* with dmrg_profile on: the contraction launches of
                             the products (kernel and chunk reduction)        */
  double split_ms;        /* with dmrg_profile on: their psi splits (tcgen05)  */
  int64_t contraction_launches;
} dmrg_bond_result;

/*
 * dmrg_bond_solve -- Davidson (Sec. II.D) for the two-site wavefunction of
 * `bond` on the blocks the context holds, from the wavefunction predicted
 * from the neighbouring bond, with the H_eff psi product in `precision`
 * (DMRG_FP64, DMRG_SPLIT_HPSI or DMRG_SPLIT_HPSI_TC), at most max_iter
 * iterations to residual tol.  Nothing of the stored state changes (no
 * decimation), so calls with different precisions start from the same
 * vector.  Every product is timed with CUDA events on the library's stream;
 * when Davidson stops before min_calls products, H_eff psi is applied to its
 * vector until min_calls have run.  call_ms (cap values, may be NULL with
 * cap 0) receives the time of each product.  direction: the direction of
 * the partial sweep that stopped next to `bond` (0 L->R, 1 R->L).
 * DMRG_ESTATE when the blocks of `bond` are not held.
 */
dmrg_status dmrg_bond_solve(dmrg_ctx* ctx, int bond, int direction, int precision, int max_iter,
                            double tol, int min_calls, int check64, dmrg_bond_result* out,
                            double* call_ms, int cap);

/*
 * dmrg_bond_apply -- y = H_eff x (Sec. II.B, the two-site effective
 * Hamiltonian without e_core) on the blocks of the last dmrg_bond_solve, in
 * the given precision (as for dmrg_bond_solve; the schedule is the default
 * one).  x and y: host vectors of *len doubles in the two-site layout of that
 * bond (the layout of its Davidson vector).  With x or y NULL only *len is
 * set to the dimension; a *len that differs from it returns DMRG_EINVAL with
 * *len set.  DMRG_ESTATE without a bond solve since the last sweep.  For
 * inspection: Hermiticity, linearity, products on chosen vectors.
 */
dmrg_status dmrg_bond_apply(dmrg_ctx* ctx, int precision, const double* x, double* y, int64_t* len);

/*
 * dmrg_bond_check64 -- the float64 Rayleigh quotient (+ e_core) and
 * residual ||H_eff psi - E psi|| (||psi|| = 1) of the vector of the last
 * dmrg_bond_solve, from one float64 H_eff psi on the same blocks; *ms its
 * CUDA-event time and *flops its algorithmic FLOPs.  dmrg_bond_solve with
 * check64 = 1 runs it and fills energy_rq64 / residual64 (0 otherwise).
 * DMRG_ESTATE without a bond solve since the last sweep.  Any NULL output is
 * skipped.
 */
dmrg_status dmrg_bond_check64(dmrg_ctx* ctx, double* energy_rq64, double* residual64, double* ms,
                              double* flops);

/* Change the Davidson iteration cap (per bond) and residual tolerance used
 * by subsequent sweeps (Sec. II.D).  A bond that reaches the cap keeps its
 * last Ritz vector. */
dmrg_status dmrg_set_davidson(dmrg_ctx* ctx, int max_iter, double tol);

/* Bound (seconds) of the device-side waits of the context's kernels for
 * subsequent calls (the wait_timeout_s option): 0 makes a wait that is not
 * complete at its first probe give up, so the call returns DMRG_ETIMEOUT and
 * the context stays usable.  DMRG_EINVAL outside [0, 3600]. */
dmrg_status dmrg_set_wait_timeout(dmrg_ctx* ctx, double seconds);

/* The same bound, process-wide, for the kernel-level entry points
 * (dmrg_hpsi_contract, dmrg_eigh_batched and the CAS-SCF routines) called
 * after it; default 2 s. */
dmrg_status dmrg_set_kernel_wait_timeout(double seconds);

/* tc_drain_terms (see dmrg_opts) of the kernel-level dmrg_hpsi_contract,
 * process-wide; default 1024. */
dmrg_status dmrg_set_kernel_tc_drain_terms(int terms);

/*
 * Schedules of the batched tcgen05 H_eff psi launch (Sec. II.B products, all
 * sector blocks of one product in one persistent launch).  A schedule is
 * {tile width N of the 128 x N sigma tiles, item chunks per CTA, task order
 * (0: longest cluster task first onto the least-loaded cluster; 1: sigma
 * block by sigma block), CTAs per cluster (2 or 4: column tiles of one row
 * tile grouped that many at a time share stage 1)}.  dmrg_tc_shape_candidates
 * writes the candidates the autotuner times, the default first, as groups of
 * four ints into shapes (room for cap groups; *count receives their number).
 */
dmrg_status dmrg_tc_shape_candidates(int* shapes, int cap, int* count);

/* Schedule candidate (index into dmrg_tc_shape_candidates) of the kernel-level
 * dmrg_hpsi_contract with DMRG_SPLIT_HPSI_TC (process-wide; default 0). */
dmrg_status dmrg_set_kernel_tc_shape(int candidate);

/* Turns the autotuning of tc_autotune (see dmrg_opts) on or off for a
 * context; tuned schedules already found stay cached. */
dmrg_status dmrg_set_tc_autotune(dmrg_ctx* ctx, int on);

/* The schedule of the last planned tcgen05 H_eff psi launch of ctx: shape[4]
 * as above; ms[k] (k < min(cap, *count)) the CUDA-event time in ms of one
 * product under candidate k for that product's sector histogram (-1: not
 * timed, or autotuning off).  DMRG_ESTATE before the first tcgen05 product. */
dmrg_status dmrg_tc_schedule_info(const dmrg_ctx* ctx, int* shape, double* ms, int cap, int* count);

/* Change the bond dimension used by subsequent sweeps. */
dmrg_status dmrg_set_bond_dim(dmrg_ctx* ctx, int D);

/* Change the GEMM precision used by subsequent sweeps (dmrg_precision). */
dmrg_status dmrg_set_precision(dmrg_ctx* ctx, int precision);

/* Energy of the last sweep (incl. e_core).  DMRG_ESTATE before any sweep. */
dmrg_status dmrg_energy(const dmrg_ctx* ctx, double* energy);

/*
 * dmrg_rdm12 -- spin-free one- and two-particle reduced density matrices of
 * the state left by the last sweep (Sec. II.C, Eqs. onerdm, twordm):
 *   gamma[p*n + q]               = <sum_s a+_{p s} a_{q s}>
 *   Gamma[((p*n + q)*n + r)*n + s] = <sum_{s,t} a+_{p s} a+_{q t} a_{r t} a_{s s}>
 * (row-major n x n and n^4, caller-allocated host buffers).  The state is
 * the two-site wavefunction of the final bond (bond 1 after a full sweep),
 * evaluated exactly in float64 by a measurement pass over all bonds (the
 * SU(2) channels Gamma^(0), Gamma^(1) of the paper are recoupled into the
 * spin-free form internally; Gamma~ = sqrt(3) Gamma^(1) - Gamma^(0) in the
 * Clebsch-Gordan convention used here).  DMRG_ESTATE before any sweep or if
 * the last sweep did not end at bond 1; DMRG_EINVAL for NULL buffers.
 */
dmrg_status dmrg_rdm12(dmrg_ctx* ctx, double* gamma, double* Gamma);

/*
 * Orbital entanglement for the orbital-ordering step (Sec. II "Numerical
 * procedure": a few low-D runs give the ordering from quantum-information
 * measures of the state).  Same state and preconditions as dmrg_rdm12.
 *
 * dmrg_orbital_rdms -- one- and two-orbital reduced density matrices,
 * averaged over the 2S+1 states of the multiplet (the SU(2)-invariant
 * reduced states).  Local states of one orbital d = 2 n_up + n_dn (0 empty,
 * 1 down, 2 up, 3 doubly occupied), the doubly occupied one a+_up a+_dn|0>.
 *   rho1[4p + d]                    weight of local state d of orbital p
 *   rho2[(p*n + q)*256 + 16 a + b]  for p < q: the 16 x 16 rho_pq over the
 *       local states a = 4 d_p + d_q (creators applied in the order p-up,
 *       p-dn, q-up, q-dn), defined by Tr(rho_pq X) = <X> for every operator
 *       X of those four modes; entries with p >= q are set to zero.
 * Host buffers of n*4 and n*n*256 doubles.  A measurement pass over all
 * bonds evaluates, in float64 on the device, the expectation values of the
 * number and double-occupancy strings of every orbital and of 15 coupled
 * products [X_p (x) Y_q]^0 per pair (see dmrg_orbital_rdms_from_invariants);
 * rho_pq follows from them exactly.
 */
dmrg_status dmrg_orbital_rdms(dmrg_ctx* ctx, double* rho1, double* rho2);

/*
 * dmrg_orbital_entanglement -- von Neumann entropies s1[p] = -Tr rho_p ln rho_p
 * and the mutual information mutual[p*n + q] = s_p + s_q - s_pq (natural
 * logarithm, zero diagonal) of the same reduced states; the spectra of all
 * rho_pq come from one batched float64 eigensolver launch.
 */
dmrg_status dmrg_orbital_entanglement(dmrg_ctx* ctx, double* s1, double* mutual);

/*
 * dmrg_orbital_rdms_from_invariants -- host-only: the reduced density
 * matrices of dmrg_orbital_rdms from the expectation values they are built
 * from.  Single-orbital strings S_0..S_8 (spinors a+ and a~ of one orbital,
 * a+(+1/2) = a+_up, a+(-1/2) = a+_dn, a~(+1/2) = a_dn, a~(-1/2) = -a_up,
 * coupled left to right with Clebsch-Gordan coefficients to the listed
 * doubled intermediate ranks):
 *   S_0 a+   S_1 a~   S_2 [a+ a~]^0   S_3 [a+ a~]^1   S_4 [a+ a+]^0
 *   S_5 [a~ a~]^0   S_6 [[a+ a+]^0 a~]^1/2   S_7 [[a~ a~]^0 a+]^1/2
 *   S_8 [[[a+ a+]^0 a~]^1/2 a~]^0.
 *   inv1[2p + t]  = <S_2 of p> (t = 0), <S_8 of p> (t = 1)
 *   inv2[(p*n + q)*15 + mu] (p < q) = <[S_a of p (x) S_b of q]^0> for
 *       (a, b) = (2,2) (2,8) (8,2) (8,8) (3,3) (0,1) (0,7) (6,1) (6,7)
 *                (1,0) (1,6) (7,0) (7,6) (4,5) (5,4), mu in that order.
 * These 15, the four single-orbital scalars and the identity span the
 * operators of two orbitals that commute with their spin and particle
 * number; rho_pq is the member of that span with these expectation values.
 */
dmrg_status dmrg_orbital_rdms_from_invariants(int n, const double* inv1, const double* inv2, double* rho1,
                                              double* rho2);

/*
 * dmrg_fiedler_order -- orbital ordering from the mutual information (the
 * ordering of Sec. II "Numerical procedure"): the orbitals sorted by the
 * Fiedler vector (eigenvector of the second-smallest eigenvalue, float64 on
 * the device) of the graph Laplacian diag(I 1) - I, the minimiser of
 * sum_pq I_pq (x_p - x_q)^2 over unit vectors orthogonal to the constant
 * vector.  order[k] = orbital placed at site k; oriented so that order[0] <
 * order[n-1]; equal components keep index order.  mutual: n x n symmetric
 * host array (its diagonal is ignored); DMRG_EINVAL if it is not finite or
 * not symmetric.  A degenerate second eigenvalue (e.g. a graph of separate
 * components) leaves the order undetermined within that eigenspace.
 */
dmrg_status dmrg_fiedler_order(const double* mutual, int n, int* order, int device);

/*
 * Statistics of the last sweep: total H_eff psi FLOPs (algorithmic, 2mnk per
 * product), time spent in H_eff psi (s), number of H_eff psi calls, total
 * Davidson iterations and the sweep wall time (s).  NULL outputs are skipped.
 */
dmrg_status dmrg_last_sweep_stats(const dmrg_ctx* ctx, double* hpsi_flops, double* hpsi_seconds,
                                  int* hpsi_calls, int* davidson_iters, double* sweep_seconds);

/* Bond energies (incl. e_core) of every optimised bond so far, in order.
 * *count receives the number available; at most cap values are written. */
dmrg_status dmrg_bond_energies(const dmrg_ctx* ctx, double* out, int cap, int* count);

/* Multiplet counts of the left blocks L(m), m = 0..n (-1 where not held). */
dmrg_status dmrg_block_dims(const dmrg_ctx* ctx, int* left, int* right);

/* The same blocks counted in U(1) states: every multiplet of spin S counts
 * 2S+1.  This is the U(1) bond dimension D~ that the paper reports beside D
 * (Sec. II.C; the D~ columns of Tables exetime and exetime-fe2s2), the
 * dimension a calculation without spin adaptation needs for the same
 * basis.  -1 where no block is held. */
dmrg_status dmrg_block_dims_u1(const dmrg_ctx* ctx, int* left, int* right);

/* Turn per-launch CUDA-event timing of the GEMM kernels on (1) or off (0);
 * turning it on resets the counters. */
dmrg_status dmrg_profile(dmrg_ctx* ctx, int on);

/* Device time (ms), algorithmic FLOPs and launch count of the GEMM kernels
 * since profiling was turned on.  which = 1: the H_eff psi contraction
 * launches (the kernel and the reduction of its item chunks), 0: all other
 * GEMM launches (renormalisation, complementary operators, density
 * matrices), 2: the blocking placement kernel, 3: the eigensolver of a single
 * small matrix (the Davidson subspace problem), 4: the batched eigensolver
 * (the density-matrix sectors of a decimation, one cooperative launch per
 * batch), 5: the TF32 hi/lo splits of the tcgen05 path's operands. */
dmrg_status dmrg_kernel_stats(dmrg_ctx* ctx, int which, double* ms, double* flops,
                              int64_t* launches);

/* Wall time (s) of the phases of the last sweep: [0] blocking (enlarged
 * operators), [1] H_eff psi task planning, [2] Davidson, [3] decimation,
 * [4] renormalisation, [5] wavefunction prediction; parts of [0]: [6] host
 * term lists, [7] host placement lists, [8] complementary-operator GEMMs,
 * [9] placement submission (grouping, upload, launch), [10] operator
 * allocation; parts of [1]: [11] host item lists, [12] task lists,
 * [13] uploads and operand splits, [14] preconditioner diagonal.
 * t must hold 15 values. */
dmrg_status dmrg_last_sweep_phases(const dmrg_ctx* ctx, double* t);

/* Device time of the last sweep in milliseconds, measured with CUDA events
 * recorded on the library's stream at the start and the end of the sweep. */
dmrg_status dmrg_last_sweep_device_ms(const dmrg_ctx* ctx, double* ms);

/* Device memory held by the context now and at its high-water mark (bytes). */
dmrg_status dmrg_memory(const dmrg_ctx* ctx, int64_t* in_use, int64_t* peak);

/* Staging detail (bytes), out[7]: [0] stored blocks on the device, [1] stored
 * blocks staged out to pinned host memory, [2] total moved out and [3] total
 * moved back in so far, [4] the largest working memory of a bond beyond the
 * stored blocks so far, [5] the largest stored block, [6] the MPS tensors
 * (kept eigenvectors of every bond, always on the device).  With hbm_budget_bytes
 * set, stored blocks whose next use in the sweep is farthest away are copied
 * to pinned host memory on a side stream whenever the stored blocks plus the
 * last bond's working memory would exceed the budget, and are copied back
 * one bond ahead of their use; the values are bit-identical either way. */
dmrg_status dmrg_memory_detail(const dmrg_ctx* ctx, int64_t* out);

/* Number of device kernel launches issued by the context so far. */
dmrg_status dmrg_launch_count(const dmrg_ctx* ctx, int64_t* launches);

/* Release every resource of the context (NULL is accepted). */
void dmrg_free(dmrg_ctx* ctx);

/* Message of the last error of ctx, or of the calling thread if ctx is NULL. */
const char* dmrg_last_error(const dmrg_ctx* ctx);

/* ------------------------------------------------------------------------
 * Kernel-level entry points (host buffers in, host buffers out).  They run
 * one launch of the device primitives the sweep is made of, so the kernels
 * can be checked element by element against a plain CPU evaluation.
 * ---------------------------------------------------------------------- */

/* One segment of a grouped GEMM: C_g += alpha * op(A) * op(B), where op(A) is
 * m x k (trans_a: A stored k x m) and op(B) is k x n (trans_b: B stored n x k).
 * Offsets are element offsets into the A / B host arrays; lda/ldb are the
 * row lengths of the stored matrices. */
typedef struct {
  int64_t a_off, b_off;
  int k, lda, ldb, trans_a, trans_b;
  double alpha;
} dmrg_gemm_seg;

/* Output block g: rows m, cols n at element offset c_off of C with row length
 * ldc; its segments are seg[seg_begin .. seg_begin + seg_count). */
typedef struct {
  int64_t c_off;
  int m, n, ldc, seg_begin, seg_count;
} dmrg_gemm_group;

/*
 * dmrg_grouped_gemm -- the segment-sum GEMM used by H_eff psi (the contraction
 * sigma = sum_t c_t A_t psi B_t^T of Sec. II.B, one output sector block per
 * group), by renormalisation and by the complementary-operator contractions.
 * C (c_len doubles) is read and updated in place; A and B are read only.
 * Output blocks must not overlap.  precision: DMRG_FP64 or DMRG_SPLIT_TF32.
 * Returns DMRG_EINVAL for out-of-range offsets, DMRG_ECUDA without a device.
 */
dmrg_status dmrg_grouped_gemm(const double* A, int64_t a_len, const double* B, int64_t b_len,
                              double* C, int64_t c_len, const dmrg_gemm_group* groups,
                              int n_groups, const dmrg_gemm_seg* segs, int n_segs, int precision,
                              int device);

/* One item of the fused H_eff psi contraction: alpha * op(A) * P * op(B)^T
 * with op(A) m x ka (trans_a: A stored ka x m), P ka x kb (row length ldp) and
 * op(B)^T kb x n (trans_b = 0: B stored n x kb; trans_b = 1: B stored kb x n).
 * a_identity / b_identity replace A / B by the identity (offsets ignored). */
typedef struct {
  int64_t a_off, p_off, b_off;
  int lda, ldp, ldb, trans_a, trans_b, ka, kb, a_identity, b_identity;
  double alpha;
} dmrg_hpsi_item;

/* Output block: rows m, cols n at c_off (row length ldc); its items are
 * item[item_begin .. item_begin + item_count). */
typedef struct {
  int64_t c_off;
  int m, n, ldc, item_begin, item_count;
} dmrg_hpsi_block;

/*
 * dmrg_hpsi_contract -- one launch of the fused H_eff psi kernel:
 *   C_block += sum_items alpha op(A) P op(B)^T   (Sec. II.B: the two-block
 * effective Hamiltonian sigma = sum_t c_t A_t psi B_t^T over sector blocks),
 * with the intermediate A P kept on chip and item chunks reduced in a fixed
 * order.  Host buffers in/out (C updated in place); all offsets are checked
 * against the buffer lengths before any launch.  precision: DMRG_FP64,
 * DMRG_SPLIT_TF32 (3xTF32 on mma.sync, 64 x 64 tiles) or DMRG_SPLIT_HPSI_TC
 * (3xTF32 on tcgen05, 128 x 64 tiles; DMRG_ETIMEOUT if a bounded wait ran
 * out).
 */
dmrg_status dmrg_hpsi_contract(const double* A, int64_t a_len, const double* P, int64_t p_len,
                               const double* B, int64_t b_len, double* C, int64_t c_len,
                               const dmrg_hpsi_block* blocks, int n_blocks,
                               const dmrg_hpsi_item* items, int n_items, int precision,
                               int device);

/* Device time (ms, CUDA events on the library's stream) of the kernels of
 * the calling thread's last dmrg_hpsi_contract: the contraction and the
 * reduction of item chunks (the operand splits of the tcgen05 path and the
 * host copies are not included). */
dmrg_status dmrg_last_contract_ms(double* ms);

/*
 * dmrg_hpsi_contract_noalloc -- the fused H_eff psi contraction of
 * dmrg_hpsi_contract on caller-owned DEVICE buffers, allocating nothing.
 * The paper has no counterpart: this entry exists for callers that cannot
 * allocate device memory while they run -- latency-critical loops where a
 * cudaMalloc or cudaFree would synchronise the device, and callers whose
 * device memory is owned by another allocator (e.g. PyTorch's caching
 * allocator, or a fixed arena set aside by a serving process), where a
 * private allocation would fragment or overcommit that memory.
 *
 * dA, dP, dB, dC: device pointers (lengths a_len .. c_len in doubles) on
 * `device`; dC is updated in place.  blocks / items: host arrays, same meaning
 * as for dmrg_hpsi_contract; every offset is checked against the lengths
 * before anything is enqueued.  The call copies the task lists to a static
 * device scratch of 32 MiB (file-scope __device__ array, one per device) and
 * enqueues the copies and the kernels on `stream` (a cudaStream_t; NULL: the
 * legacy default stream); it returns without synchronising.  A request whose
 * task lists and partial tiles exceed the 32 MiB returns DMRG_EINVAL with the
 * size it needed (use dmrg_hpsi_contract for it).  precision: DMRG_FP64 or
 * DMRG_SPLIT_TF32.  Nothing in the scratch has to start at zero: every
 * partial tile is written in full before the reduction reads it.
 *
 * The scratch is shared by all calls on a device: calls that overlap in time
 * (two host threads, or two streams whose work is in flight together) race
 * on it and give wrong results; serialise them.  The first call on a device
 * looks up the scratch address (cudaGetSymbolAddress, with that device made
 * current and then restored) and sets the kernels' shared-memory attributes
 * for that device.  The task lists are copied from host memory that lives
 * only for the duration of the call, so the entry is for eager calls:
 * recording it into a CUDA graph by stream capture is not supported.
 */
dmrg_status dmrg_hpsi_contract_noalloc(const double* dA, int64_t a_len, const double* dP, int64_t p_len,
                                       const double* dB, int64_t b_len, double* dC, int64_t c_len,
                                       const dmrg_hpsi_block* blocks, int n_blocks,
                                       const dmrg_hpsi_item* items, int n_items, int precision,
                                       int device, void* stream);

/*
 * dmrg_eigh_batched -- symmetric eigendecompositions in float64 on the device
 * (the sector density matrices of the decimation step, Sec. II.C).  mats holds
 * the row-major matrices back to back (sizes n[i]); w receives eigenvalues in
 * descending order and vecs the eigenvectors as rows (same packing as mats).
 * Largest-magnitude component of every eigenvector is made positive.
 */
dmrg_status dmrg_eigh_batched(const double* mats, const int* n, int count, double* w, double* vecs,
                              int device);

/* ------------------------------------------------------------------------
 * CAS-SCF side (Sec. II.A).  Orbitals are ordered core (ncore), active
 * (ncas), virtual (the rest); nb is the total number of orbitals.  Cholesky
 * vectors chol[k, p, q] = L^k_pq give (pq|rs) = sum_k L^k_pq L^k_rs.
 * Host arrays in and out, float64 row-major; all arithmetic on the device.
 * ---------------------------------------------------------------------- */

/* Device time (ms, CUDA events on the call's stream) and algorithmic FLOPs
 * (2mnk per product) of the grouped float64 GEMM launches of the calling
 * thread's last casscf_* call: for casscf_transform these are all of its
 * arithmetic (the host copies are not included). */
dmrg_status casscf_last_kernel_ms(double* ms, double* flops);

/* R = expm(-K) for the real antisymmetric K with K[p,q] = kappa_pq (p > q):
 * U = exp(-kappa^) of Sec. II.A rotates the integrals as h' = R^T h R. */
dmrg_status casscf_rotation(const double* K, int nb, double* R, int device);

/* Backward of R = expm(-K): given G = dE/dR (nb x nb) return the
 * antisymmetric dK with dK[p,q] = dE/dkappa_pq (p > q), dK[q,p] = -dK[p,q]
 * (adjoint Frechet derivative of the exponential, via the 2nb x 2nb block
 * exponential). */
dmrg_status casscf_rotation_backward(const double* K, const double* G, int nb, double* dK,
                                     int device);

/* Integral transformation: h_out = R^T h R, chol_out[k] = R^T chol[k] R. */
dmrg_status casscf_transform(const double* R, const double* h, const double* chol, int rank,
                             int nb, double* h_out, double* chol_out, int device);

/* Active-space problem handed to DMRG: e_core (closed-shell core energy),
 * h_act = inactive Fock matrix on the active block (ncas x ncas) and
 * eri_act = (tu|vw) of the active orbitals (ncas^4). */
dmrg_status casscf_active_space(const double* h, const double* chol, int rank, int nb, int ncore,
                                int ncas, double* e_core, double* h_act, double* eri_act,
                                int device);

/* Orbital gradient at the current orbitals (kappa = 0) from the spin-free
 * RDMs of the active space (gamma: ncas^2; Gamma: ncas^4 in the operator
 * order of Eq. twordm):  grad = 2 (F - F^T) with the generalised Fock matrix
 * F (textbook closed-shell-core form), grad[p,q] = dE/dkappa_pq for p > q,
 * active-active block zero (those rotations are not used, Sec. II.C).
 * fock (optional, may be NULL) receives F. */
dmrg_status casscf_orbital_gradient(const double* h, const double* chol, int rank, int nb,
                                    int ncore, int ncas, const double* gamma, const double* Gamma,
                                    double* grad, double* fock, int device);

/*
 * casscf_transform_backward -- backward of the map kappa -> (e_core, h_act,
 * eri_act) = casscf_active_space(casscf_transform(expm(-K), h, chol)) of
 * Sec. II.A, for upstream weights g_core (scalar), g_h (ncas^2) and g_eri
 * (ncas^4): the weighted sum is a CAS-SCF energy functional with RDMs
 * gamma = sym(g_h) / g_core and Gamma_tvwu = 2 sym8(g_eri)_tuvw / g_core, its
 * derivative with respect to the rotated orbitals is dE/dR = 2 R F^T (F the
 * generalised Fock matrix of casscf_orbital_gradient in the rotated basis;
 * with g_core = 0 the core part of F is subtracted), and the adjoint Frechet
 * derivative of expm carries it to K.  K: the antisymmetric nb x nb input,
 * R = expm(-K), h_rot / chol_rot: the rotated integrals of the forward call.
 * dK receives dE/dK, the gradient with respect to the full antisymmetric
 * matrix (half of dE/dkappa_pq on both (p,q) and (q,p) with opposite signs).
 */
dmrg_status casscf_transform_backward(const double* K, const double* R, const double* h_rot,
                                      const double* chol_rot, int rank, int nb, int ncore, int ncas,
                                      double g_core, const double* g_h, const double* g_eri, double* dK,
                                      int device);

/* Options of the DMRG-SCF macro iterations. */
typedef struct {
  int max_iter;     /* macro iterations (60)                                 */
  double e_tol;     /* energy change of the last iteration (1e-7 Eh)         */
  double g_tol;     /* largest orbital-gradient entry (1e-3)                 */
  int memory;       /* L-BFGS pairs kept (8)                                 */
  double max_step;  /* cap of the largest rotation entry of a step (0.5)     */
  int sweeps;       /* DMRG sweeps per macro iteration (4)                   */
} casscf_scf_opts;

void casscf_default_scf_opts(casscf_scf_opts* o);

/*
 * casscf_dmrg_scf -- the DMRG-SCF macro loop of Sec. II.A (the paper's
 * thresholds: 1e-7 in the energy, 1e-3 in the orbital gradient).  Per
 * iteration: the integrals rotated by the accumulated orbital rotation U
 * (casscf_transform), the active-space problem (casscf_active_space), a
 * DMRG-CI solve of it (dmrg_opts; `sweeps` sweeps from the default product
 * state) and its spin-free RDMs (dmrg_rdm12), the orbital gradient
 * (casscf_orbital_gradient) and a step: limited-memory BFGS over the
 * non-redundant rotations (core-active, core-virtual, active-virtual) with
 * an approximate diagonal Hessian (virtual-core 4 (f_a - f_i), virtual-active
 * 2 n_t f_a - 2 F_tt, active-core 4 (f_t - f_i) + 2 n_t f_i - 2 F_tt, f =
 * F^I + F^A, floored at 0.05) as the initial inverse and the largest entry
 * capped at max_step; U <- U expm(-(x - x^T)).  Stops after an iteration
 * whose energy changed by less than e_tol with max |g| below g_tol.
 * Outputs: U (nb x nb), energies and gmax (max_iter values, the first
 * *n_iter written), *converged (1 or 0).  ORCA's SuperCI(PT) optimiser of
 * the paper is not part of this library.
 */
dmrg_status casscf_dmrg_scf(const double* h, const double* chol, int rank, int nb, int ncore, int ncas,
                            int n_elec, int two_s, const dmrg_opts* dopts, const casscf_scf_opts* sopts,
                            double* U, double* energies, double* gmax, int* n_iter, int* converged);

#ifdef __cplusplus
}
#endif
#endif /* DMRGSCF_H */
