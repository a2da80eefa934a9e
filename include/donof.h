/*
 * donof.h -- C ABI of the GB300 library for the PNOF5 / PNOF7 / PNOF7s energy and
 * orbital-Lagrangian build (one "build" = E, lambda, dE/dgamma for one set of
 * natural orbitals C and occupation variables gamma).
 *
 * What is computed (paper sections and equations of arXiv:2004.06142):
 *   occupations n_p(gamma) ............ Sec. III.A, Eqs. soo, woo
 *   J_pq, K_pq (L = K, real orbitals) . Sec. III.D, Eqs. JKpq, Gpmn, with
 *                                       density-fitted integrals
 *                                       (mu nu|eta delta) = sum_P B[P][mu][nu] B[P][eta][delta]
 *   E ................................. Sec. II, Eqs. EPNOF7, Eg, Efg (PNOF7), Efg with
 *                                       Phi = 0 (PNOF5), Sec. V Eq. Efg_s (PNOF7s)
 *   lambda_qp = n_p H_qp + g_pq ....... Sec. III.B, Eqs. lowdin, Vee-s, Vee-d, lag, gval,
 *                                       normalised so that lambda = C^T G with
 *                                       G = (1/4) dE/dC (Eq. lowdin carries the 4)
 *   dE/dgamma, dE/dC .................. derivatives of the energy above
 *
 * Conventions shared by every entry point
 *   - Every array is row-major.  Floating point arrays are IEEE double.
 *   - Pointers marked (device) must be CUDA device pointers on the current device;
 *     pointers marked (host) are host pointers.  The library never frees caller memory.
 *   - h[nbf*nbf]   one-electron matrix, symmetric.
 *   - B            DONOF_B_DENSE : [naux][nbf][nbf], each slice symmetric;
 *                  DONOF_B_PACKED: [naux][nbf*(nbf+1)/2], element (mu >= nu) at
 *                                  mu*(mu+1)/2 + nu.
 *   - C[nbf*nbf]   MO coefficients, column p is orbital p (Eq. lcao): C[mu*nbf + p].
 *   - gamma[npair*ncwo]  gamma[0..npair) strong (Eq. soo), then (ncwo-1) weak gammas
 *                  per pair, pair-major (Eq. woo).
 *   - pair_map[nact], nact = npair*(1+ncwo) + nsingle <= nbf: subspace of each active
 *                  orbital.  pair_map[g] == g for g < npair (strong orbital g sits at
 *                  index g) and for the nsingle singly occupied orbitals of a multiplet
 *                  (Omega_I, Sec. II) at npair <= g < npair + nsingle, each its own
 *                  subspace with n = 1/2; every pair owns exactly ncwo weak orbitals with
 *                  index >= npair + nsingle; the weak orbitals of a pair, in increasing
 *                  index, are p_1..p_Ng of Eq. woo.  Orbitals p >= nact are empty (n_p = 0).
 *   - lam[nbf*nbf] lam[q*nbf + p] = lambda_qp (column p is the differentiated orbital);
 *                  columns p >= nact are zero.
 *   - Calls are asynchronous on `stream` (a cudaStream_t, 0 = legacy default stream).
 *   - Return value: DONOF_OK (0) or a negative DONOF_ERR_* code; on error the outputs
 *     are undefined.  Checks that need device data (pair_map contents, non-finite
 *     inputs, kernel wait limits) write a status word into the workspace that
 *     donof_read_status() returns.
 *   - Workspace: caller-allocated device memory of donof_workspace_size() bytes,
 *     256-byte aligned.  A workspace belongs to one problem description; the forward
 *     state that donof_energy_backward() and donof_get_jk() read lives there, so those
 *     calls must use the same workspace and stream as the forward call.  Calls that
 *     share a workspace must not overlap in time.
 */
#ifndef DONOF_H
#define DONOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { DONOF_PNOF5 = 5, DONOF_PNOF7 = 7, DONOF_PNOF7S = 8 };
enum { DONOF_B_DENSE = 0, DONOF_B_PACKED = 1 };
/* DONOF_FP64: every contraction in IEEE double on the CUDA cores.
 * DONOF_MIXED: the large contractions (X = B C, b = C^T X, G += X Y, lambda = C^T G) on the
 * tensor cores.  Every operand row is stored as 2^e (h + f): h an fp16 integer with the
 * row's L2 norm bounding ||h||_2 below 2^12, f the fp16 remainder.  The integer products
 * h*h then accumulate exactly in fp32 (no partial sum reaches 2^24), and h*f + f*h + f*f
 * go to a second accumulator.  h C_act and lambda = C^T G take each operand's split
 * extended by its residual r = y - h - f (fp16), the product cut into four K blocks kept
 * apart until a double sum: about 1e-10 relative to the row norms.  The
 * energy and dE/dgamma are in double; J, K and G are summed over slices in short fp32
 * groups (16 slices for J and K, 8 split partials for G) and in double across groups.
 * The tensor-core outputs pass through fp32, so the mixed path needs each product of two
 * operand row norms (e.g. a row of h times a column of C) between about 1e-30 and 1e30. */
enum { DONOF_FP64 = 0, DONOF_MIXED = 1 };

enum {
  DONOF_OK = 0,
  DONOF_ERR_INVALID_ARG = -1,   /* bad size, null pointer, unknown enum */
  DONOF_ERR_PAIR_MAP = -2,      /* pair_map violates the layout rules above */
  DONOF_ERR_NONFINITE = -3,     /* gamma or a reduced quantity is NaN / Inf */
  DONOF_ERR_WORKSPACE = -4,     /* workspace too small or misaligned */
  DONOF_ERR_CUDA = -5,          /* a CUDA runtime / driver call failed */
  DONOF_ERR_TIMEOUT = -6,       /* a bounded device-side wait ran out */
  DONOF_ERR_UNSUPPORTED = -7,   /* shape outside the supported range (e.g. nact > 256 mixed) */
  DONOF_ERR_NOT_PREPARED = -8   /* donof_prepare_B was not called for this workspace / B */
};

typedef struct {
  int32_t nbf;         /* N_B, number of AO basis functions, >= 1 */
  int32_t naux;        /* number of auxiliary (fitting) functions P, >= 1 */
  int32_t npair;       /* N_II / 2, electron pairs, >= 1 */
  int32_t ncwo;        /* N_g, weak orbitals per pair, >= 1 */
  int32_t functional;  /* DONOF_PNOF5 | DONOF_PNOF7 | DONOF_PNOF7S */
  int32_t b_layout;    /* DONOF_B_DENSE | DONOF_B_PACKED */
  int32_t precision;   /* DONOF_FP64 | DONOF_MIXED */
  int32_t nsingle;     /* N_I, singly occupied orbitals of a multiplet (S = N_I / 2), >= 0:
                        * n = 1/2 each, no intra-subspace term, H_gg in E and E_fg with every
                        * other subspace (Eqs. EPNOF7, Efg / Efg_s) */
  /* Upper bound, in bytes, on the per-pass intermediate X[P][mu][q] (and its
   * companions) held in the workspace; the auxiliary index is streamed in blocks that
   * fit.  0 = hold every P at once. */
  uint64_t x_budget_bytes;
} donof_problem;

/* Bytes of device workspace needed by `prob` (writes *bytes). */
int donof_workspace_size(const donof_problem* prob, size_t* bytes);

/* Register B (device) with the workspace.  DONOF_MIXED: converts B once into the
 * integer + fraction fp16 copy that every later build streams (B is fixed across orbital
 * iterations, Sec. III.D).  DONOF_FP64: records B only.  Must be called again when B
 * changes; the build calls must then pass the same B pointer. */
int donof_prepare_B(const donof_problem* prob, const double* B, void* workspace,
                    size_t workspace_bytes, void* stream);

/* One build.  Inputs h, B, C, gamma, pair_map (device).  Outputs (device):
 * E[1], lam[nbf*nbf], dE_dgamma[npair*ncwo]; lam and dE_dgamma may be NULL. */
int donof_energy_lagrangian(const donof_problem* prob, const double* h, const double* B,
                            const double* C, const double* gamma, const int32_t* pair_map,
                            void* workspace, size_t workspace_bytes, double* E, double* lam,
                            double* dE_dgamma, void* stream);

/* Adjoint of the last build in `workspace`: given the upstream gradient Ebar (device,
 * one double), writes dE_dC[nbf*nbf] = Ebar * dE/dC = 4 Ebar G (zero columns p >= nact)
 * and dE_dgamma[npair*ncwo] = Ebar * dE/dgamma (device; either may be NULL). */
int donof_energy_backward(const donof_problem* prob, const double* Ebar, const void* workspace,
                          size_t workspace_bytes, double* dE_dC, double* dE_dgamma, void* stream);

/* One build and its adjoint for a caller whose orbitals and occupation parameters live in
 * host memory (an orbital-optimisation driver on the CPU): copies C_host[nbf*nbf] and
 * gamma_host[npair*ncwo] to the device, runs donof_energy_lagrangian and, when dE_dC_host is
 * not NULL, donof_energy_backward with Ebar = 1, copies E (and lambda, dE/dgamma, dE/dC where
 * their host pointers are not NULL) back to E_host[1], lam_host[nbf*nbf],
 * dE_dgamma_host[npair*ncwo], dE_dC_host[nbf*nbf], and waits for `stream`.  h, B, pair_map and
 * the workspace are device memory as for donof_energy_lagrangian (B prepared with
 * donof_prepare_B); `staging` is a caller-allocated device buffer of
 * donof_host_staging_size bytes (256-byte aligned) that holds the device copies.  With
 * page-locked host buffers the copies are DMA transfers at full rate.  Returns a host-side
 * error code, or else the build's device-side status (as donof_read_status, which it reads
 * and clears). */
int donof_host_staging_size(const donof_problem* prob, size_t* bytes);
int donof_energy_lagrangian_host(const donof_problem* prob, const double* h, const double* B,
                                 const double* C_host, const double* gamma_host,
                                 const int32_t* pair_map, void* workspace,
                                 size_t workspace_bytes, void* staging, size_t staging_bytes,
                                 double* E_host, double* lam_host, double* dE_dgamma_host,
                                 double* dE_dC_host, void* stream);

/* A build sharded over the auxiliary index, one shard per GPU (Sec. III.D: J_pq, K_pq of
 * Eq. JKpq and the exchange and Coulomb operators of Eq. Gpmn are sums over the auxiliary
 * functions P of the density-fitted integrals, and so is the two-electron part of the
 * generalised-Fock action G of Eqs. Vee-s, Vee-d).  Each shard holds its own slices of B
 * and describes them as a problem of its own: `prob` with naux = the slices it holds, its
 * workspace prepared with donof_prepare_B on those slices.
 *   donof_partial_size: *count (host) = 2 nact^2 + nbf nact, the doubles of one partial.
 *   donof_energy_lagrangian_partial: this shard's partial sums (device, caller-owned,
 *     partial[count]): J[nact][nact], then K[nact][nact], then the two-electron part of
 *     G[nbf][nact], each a sum over the shard's slices (FP64 path: in double; mixed path:
 *     as in donof_energy_lagrangian).
 *   (the caller sums the partials of all shards elementwise, e.g. an all-reduce)
 *   donof_energy_lagrangian_finish: from the summed partial (device) and the shard's own
 *     h, C, gamma, pair_map, forms what a full build forms after its sums over P: E,
 *     lambda, dE/dgamma (outputs as in donof_energy_lagrangian), and leaves G, J, K in the
 *     workspace, so that donof_energy_backward and donof_get_jk work after it.  It reads no
 *     B.  Every shard may finish (the results agree), or only one.
 * The summed partials reproduce a full build on all the slices up to the order of the sums
 * over P. */
int donof_partial_size(const donof_problem* prob, size_t* count);
int donof_energy_lagrangian_partial(const donof_problem* prob, const double* h, const double* B,
                                    const double* C, const double* gamma,
                                    const int32_t* pair_map, void* workspace,
                                    size_t workspace_bytes, double* partial, void* stream);
int donof_energy_lagrangian_finish(const donof_problem* prob, const double* h, const double* C,
                                   const double* gamma, const int32_t* pair_map,
                                   const double* partial, void* workspace,
                                   size_t workspace_bytes, double* E, double* lam,
                                   double* dE_dgamma, void* stream);

/* Copies J[nact*nact] and K[nact*nact] (device) of the last build in `workspace`. */
int donof_get_jk(const donof_problem* prob, const void* workspace, size_t workspace_bytes,
                 double* J, double* K, void* stream);

/* Synchronises `stream`, then returns in *status (host) the device status word of the
 * last call on `workspace` (DONOF_OK or a DONOF_ERR_* code) and clears it. */
int donof_read_status(const void* workspace, int32_t* status, void* stream);

/* Occupation optimisation at fixed orbitals (Sec. III.D: in every iteration gamma is
 * optimised for fixed natural orbitals, by CG or L-BFGS).  Minimises E[n(gamma), phi] of
 * Eqs. EPNOF7 / Eg / Efg (/ Efg_s) over the unconstrained gamma (occupations by Eqs. soo,
 * woo) with L-BFGS (memory 8) and an Armijo backtracking line search, in one CTA, using the
 * H_pp, J_pq and K_pq of the last donof_energy_lagrangian call on `workspace` (same problem;
 * the orbitals of that call are the fixed ones).  Since the occupations depend on each gamma
 * only through |sin gamma| and |cos gamma|, the search runs over the box [0, pi/2]^ng of
 * representatives (projected L-BFGS; the start point is folded into it first), so that a
 * minimum on a kink of sqrt(n) = |sin gamma| is a minimum on a bound.  gamma[npair*ncwo]
 * (device) holds the start point on entry and the optimum (in the box) on return; E (device
 * scalar, may be NULL) receives the optimal energy and iters (device int32, may be NULL) the
 * L-BFGS iterations taken.  Stops when the projected gradient is below gtol in every
 * component, when no step lowers E any further, or after max_iter iterations.  DONOF_ERR_UNSUPPORTED when nact is too large for one CTA's shared memory
 * (about 2400 active orbitals). */
int donof_optimize_occupations(const donof_problem* prob, const int32_t* pair_map,
                               double* gamma, void* workspace, size_t workspace_bytes,
                               int32_t max_iter, double gtol, double* E, int32_t* iters,
                               void* stream);

/* Hand-off to the orbital update (Sec. III.B).  Builds the symmetric matrix of Eq. Fockian,
 *   F_qp = theta(p - q)[lambda_qp - lambda_pq] + theta(q - p)[lambda_pq - lambda_qp] (q != p),
 *   F_pp = Fdiag[p]   (the paper takes the diagonal from the previous diagonalisation),
 * diagonalises it in double (donof_eigh), F = V diag(eps) V^T with eps ascending, and writes the rotated
 * orbitals C_new = C V after one double Newton-Schulz reorthonormalisation step
 * C_new <- C_new (3 I - C_new^T C_new) / 2.  lam, Fdiag[nbf], C (device, as in
 * donof_energy_lagrangian) in; C_new[nbf*nbf] (column j = new orbital j) and eps[nbf]
 * (device) out; nbf <= 4096.  Workspace: donof_orbital_update_workspace_size bytes (device,
 * 256-byte aligned).  Note: with lambda as defined here (lambda = C^T G, G = dE/dC / 4) the first-order
 * energy change of this update is 4 sum_{q<p} F_qp^2 / (F_pp - F_qq), so a diagonal that
 * decreases with the orbital index lowers E (the paper's Eq. ene1 prints the opposite sign). */
int donof_orbital_update_workspace_size(int32_t nbf, size_t* bytes);
int donof_orbital_update(int32_t nbf, const double* lam, const double* Fdiag, const double* C,
                         void* workspace, size_t workspace_bytes, double* C_new, double* eps,
                         void* stream);

/* Symmetric eigendecomposition in double: the diagonalisation step of Sec. III.B (the new
 * orbitals are the eigenvectors of the symmetric F of Eq. Fockian; donof_orbital_update and
 * donof_optimize call it).  A = V diag(w) V^T with w ascending.
 *   A[n*n]: device, row-major, symmetric (both triangles are read and must agree); not
 *           modified.
 *   V[n*n]: device, row-major, column j = eigenvector j (unit norm); may be A's buffer.
 *   w[n]:   device, eigenvalues in ascending order.
 * 1 <= n <= 4096.  Workspace: donof_eigh_workspace_size(n) bytes of device memory, 256-byte
 * aligned, owned by the caller (one call at a time per workspace).  Method: Householder
 * reduction to tridiagonal T in one cooperative launch (one CTA per SM); T split where an
 * off-diagonal element is at most 16 n eps ||T||_inf; eigenvalues by bisection on Sturm
 * counts; eigenvectors of T from twisted factorisations, and by inverse iteration with
 * block orthonormalisation for eigenvalues of one block closer than 1e-5 ||T||_inf (every
 * member's own inverse iteration; clusters of more than 32 members in panels on the GEMM
 * kernel); V = Q Z in blocks of 64 reflectors.  The call waits once for `stream` (after the
 * eigenvalues, to read the clusters' layout on the host), so it cannot be captured into a
 * CUDA graph; donof_orbital_update and donof_optimize inherit that wait.  Each eigenvalue is
 * within a small multiple of n eps ||A|| of the exact one and each eigenvector within that
 * over its gap; columns of V are orthonormal to about n eps ||A|| / (smallest gap outside the
 * clusters).
 * Returns DONOF_ERR_INVALID_ARG (n out of range, NULL pointer), DONOF_ERR_WORKSPACE, or
 * DONOF_ERR_CUDA (a failed launch, also when the cooperative launch cannot make its grid
 * co-resident).  Device-side outcomes (A not finite; a grid-barrier wait that ran out after
 * 2 s, which leaves NaN eigenvalues) are read with donof_eigh_read_status, which waits for
 * `stream` and writes DONOF_OK, DONOF_ERR_NONFINITE or DONOF_ERR_TIMEOUT to *status. */
int donof_eigh_workspace_size(int32_t n, size_t* bytes);
int donof_eigh(int32_t n, const double* A, double* V, double* w, void* workspace,
               size_t workspace_bytes, void* stream);
int donof_eigh_read_status(const void* workspace, int32_t* status, void* stream);

/* Batched builds: ninst independent instances (e.g. one molecule at many geometries), each
 * with its own problem description probs[i] and device pointers inst[i].  The workspace
 * (donof_batched_workspace_size bytes) holds a head (the batch's status word at its start,
 * then the tables below) and one slice per instance; prepare every B once with
 * donof_prepare_B_batched.
 * When every instance is DONOF_MIXED with all its auxiliary slices in one block (no
 * x_budget_bytes split), each step of the build runs as one launch for all instances (26
 * launches per batched build and adjoint, whatever ninst): the tables that map a launch's
 * blocks and tensor-core work units to instances are built on the host and copied into the
 * workspace head when the arguments change (a synchronisation of `stream`).  Otherwise
 * instances run their single-instance sequences concurrently on library-owned streams that
 * fork from and join back to `stream`.  Both give the same results bit for bit.
 *   DONOF_BATCH_BACKWARD: also write inst[i].dE_dC = dE/dC (upstream gradient 1).
 *   DONOF_BATCH_GRAPH: capture the whole batch into a CUDA graph on the first call and
 *     replay it (one graph launch) on every later call with identical arguments (same
 *     problems, pointers, workspace and flags); tracing is not recorded inside graphs.
 *   DONOF_BATCH_STREAMS: use the per-instance streams even where the grouped launches apply.
 * Device-side checks of an instance go to its own status word (donof_read_status on its
 * slice); wait limits of the grouped tensor-core launches to the batch's (donof_read_status
 * on the workspace). */
typedef struct {
  const double* h;
  const double* B;
  const double* C;
  const double* gamma;
  const int32_t* pair_map;
  double* E;          /* [1] */
  double* lam;        /* [nbf*nbf] or NULL */
  double* dE_dgamma;  /* [npair*ncwo] or NULL */
  double* dE_dC;      /* [nbf*nbf] or NULL (DONOF_BATCH_BACKWARD) */
} donof_instance;
enum { DONOF_BATCH_BACKWARD = 1, DONOF_BATCH_GRAPH = 2, DONOF_BATCH_STREAMS = 4 };
int donof_batched_workspace_size(int32_t ninst, const donof_problem* probs, size_t* bytes);
int donof_prepare_B_batched(int32_t ninst, const donof_problem* probs, const donof_instance* inst,
                            void* workspace, size_t workspace_bytes, void* stream);
int donof_energy_lagrangian_batched(int32_t ninst, const donof_problem* probs,
                                    const donof_instance* inst, void* workspace,
                                    size_t workspace_bytes, int32_t flags, void* stream);

/* The parts of the NOF-MP2 energy (Sec. "Dynamic Correlation", Eq. Etotal:
 * E = E_hf~ + E^sta + E^dyn) that need only the integrals of a build, from the H_pp, J_pq,
 * K_pq and occupations of the last donof_energy_lagrangian call on `workspace` (same
 * problem and pair_map):
 *   E_hf  (device scalar) = Eq. HFL, the energy of its closed-shell-like HF density matrix
 *                            with 2n_g = 2 (pairs) and 2n_g = 1 (singly occupied orbitals):
 *                            2 sum_g w_g H_gg + sum_{f,g} w_f w_g (2 J_fg - K_fg)
 *                            - sum_{g singly occupied} J_gg / 4, w_g = 1 for the strong
 *                            orbital of a pair and 1/2 for a singly occupied one, f and g
 *                            over the npair + nsingle strong orbitals (indices
 *                            0 .. npair+nsingle-1); without singles, the printed formula;
 *   E_sta (device scalar) = Eq. Esta: sum over the pair subspaces and ordered q != p in each
 *                            of sqrt(Lambda_q Lambda_p) Pi_qp K_pq, Lambda_p = 1 - |1 - 2 n_p|,
 *                            minus 4 sum over ordered pairs in different subspaces of
 *                            Phi_q^2 Phi_p^2 K_pq.
 * E^dyn (Eq. E2) is not computed: its amplitudes come from modified MP2 residual equations
 * that the paper cites but does not state.  One CTA; fixed summation order. */
int donof_nofmp2_static(const donof_problem* prob, const int32_t* pair_map,
                        const void* workspace, size_t workspace_bytes, double* E_hf,
                        double* E_sta, void* stream);

/* The optimisation procedure around the build (Sec. III.D, with Sec. III.B's scaling and
 * Sec. III.C's DIIS).  Each outer iteration optimises the occupations at fixed orbitals
 * (donof_optimize_occupations) and then the orbitals at fixed occupations by up to
 * max_inner diagonalisations of F (Eq. Fockian):
 *   - the off-diagonal of F comes from the build's lambda; every element above zeta in
 *     magnitude is divided by ten until it is not (zeta <= 0: no scaling);
 *   - the diagonal is the previous diagonalisation's eigenvalues (Fdiag, in/out);
 *   - F and its error vector e = offdiag F are taken to the AO basis (C F C^T, C e C^T) and,
 *     with diis_depth >= 2, the last diis_depth of them are combined with the coefficients
 *     of the bordered least-squares system of Sec. III.C;
 *   - the eigenvectors of the result, in decreasing eigenvalue order (the energy-lowering
 *     order for lambda = C^T G as defined here), are the new orbitals, reorthonormalised by
 *     one Newton-Schulz step, and those eigenvalues the next diagonal.
 * The orbital iterations of an outer iteration stop when max |lambda_qp - lambda_pq| < delta
 * or E changed by less than eps_energy; the procedure has converged when, after an outer
 * iteration, the asymmetry is below delta and E changed by less than eps_energy over it.
 * With init_diagonal != 0 the start follows Sec. III.D's initial step: after the first
 * occupation optimisation the symmetrised lambda is diagonalised, its eigenvectors (ascending)
 * rotate C and minus its eigenvalues are the first diagonal; otherwise Fdiag is used as given.
 * h, B, pair_map as for donof_energy_lagrangian (B already prepared in build_ws); C[nbf*nbf],
 * gamma[npair*ncwo] and Fdiag[nbf] are device arrays updated in place.  opt_ws: device,
 * 256-byte aligned, donof_optimize_workspace_size bytes.  The call is synchronous: the host
 * reads E and the asymmetry after every build.  *result (host) receives the final E and
 * asymmetry, the iteration counts and whether it converged; energies (host, optional)
 * receives the energy of every orbital-iteration build, at most energies_cap of them. */
typedef struct {
  int32_t max_outer;    /* outer iterations (>= 1) */
  int32_t max_inner;    /* diagonalisations per outer iteration (>= 1) */
  int32_t diis_depth;   /* 0 or 1: no extrapolation; 2..16: matrices combined */
  int32_t occ_max_iter; /* L-BFGS iterations per occupation optimisation */
  double zeta;          /* scaling bound of F's off-diagonal (<= 0: none) */
  double delta;         /* max |lambda_qp - lambda_pq| criterion */
  double eps_energy;    /* energy criterion */
  double occ_gtol;      /* occupation optimisation: max |dE/dgamma| criterion (> 0) */
} donof_opt_params;

typedef struct {
  double E;             /* energy at the final orbitals and occupations */
  double max_asym;      /* max |lambda_qp - lambda_pq| there */
  int32_t outer, inner, builds, converged, energies_recorded, reserved;
} donof_opt_result;

int donof_optimize_workspace_size(const donof_problem* prob, int32_t diis_depth, size_t* bytes);
int donof_optimize(const donof_problem* prob, const donof_opt_params* params, const double* h,
                   const double* B, double* C, double* gamma, const int32_t* pair_map,
                   double* Fdiag, int32_t init_diagonal, void* build_ws, size_t build_bytes,
                   void* opt_ws, size_t opt_bytes, donof_opt_result* result, double* energies,
                   int32_t energies_cap, void* stream);

/* A build that allocates no device memory, for callers that cannot allocate at the time
 * they need one (a host framework that owns the device memory pool, a loop where an
 * allocation's synchronisation or failure is not acceptable).  The paper has no
 * counterpart; this is a deployment convenience.
 * Inputs h, B, C, gamma, pair_map and outputs E[1], lam (may be NULL), dE_dgamma (may be
 * NULL) and dE_dC[nbf*nbf] (= dE/dC, may be NULL) are caller-owned device pointers as in
 * donof_energy_lagrangian / donof_energy_backward; B is converted on every call (there is
 * no separate prepare step).
 * Scratch: a fixed 64 MiB array in device global memory, held by every GPU that loads the
 * library until the process exits.  Problems whose donof_workspace_size exceeds it are
 * rejected with DONOF_ERR_WORKSPACE before any device work.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current (and
 * looks it up again after a reset of the device's context); make that first call before
 * any stream capture.  Every call on a device shares the array and leaves its contents
 * behind: the call clears what must start at zero itself.  Calls from several host threads
 * on one device are serialised on the host; calls whose device work overlaps (other
 * streams) race on the array.
 * Device-side checks (pair_map contents, non-finite gamma, B, C or results, kernel wait
 * limits) write the status word at the head of the array; donof_noalloc_read_status reads
 * it.  The next call clears it, so read it before the next call.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
int donof_energy_lagrangian_noalloc(const donof_problem* prob, const double* h, const double* B,
                                    const double* C, const double* gamma,
                                    const int32_t* pair_map, double* E, double* lam,
                                    double* dE_dgamma, double* dE_dC, void* stream);

/* Synchronises `stream`, then returns in *status (host) the device status word of the last
 * donof_energy_lagrangian_noalloc call on the current device (DONOF_OK or a DONOF_ERR_*
 * code) and clears it.  Allocates nothing. */
int donof_noalloc_read_status(int32_t* status, void* stream);

/* Launch autotuner (DONOF_MIXED): times each tensor-core contraction of a build (a few builds
 * on the given inputs, B already prepared) in each of its launch variants and keeps the
 * fastest per contraction for this shape: for b = C^T X and the G contraction the K tile (64
 * or 32 elements) on single CTAs, or 256-row tiles on CTA pairs (cta_group::2); for the half
 * transform single CTAs or CTA pairs, with a grid of a whole number of slices' row tiles or of
 * every SM pair.  Later builds of the same shape use the choice.  If the environment variable
 * DONOF_TUNE_CACHE names a file, choices are loaded from it on first use and written back
 * after tuning.  Uses (and clears) the tracing record; returns DONOF_OK without work for
 * DONOF_FP64. */
int donof_autotune(const donof_problem* prob, const double* h, const double* B, const double* C,
                   const double* gamma, const int32_t* pair_map, void* workspace,
                   size_t workspace_bytes, void* stream);

/* Tracing.  While enabled, every call records a pair of CUDA events on its stream around
 * each phase of the build; donof_profile_read() waits for them and returns the summed
 * device time (ms) and the number of timed intervals of one phase.  Enabling clears the
 * previous record.  The launch counter counts every kernel the library has launched in
 * this process (tracing on or off).  Independently of tracing, each phase is also an NVTX
 * range named "donof/<phase>" (prep, half_transform, mo_3index, jk_y, g_build,
 * energy_lambda, backward, prepare_B, orbital_update, occ_opt, orbital_step) on the calling
 * host thread, for profilers that filter by range. */
enum {
  DONOF_PHASE_PREP = 0,            /* occupations, coefficients, h C, operand splits */
  DONOF_PHASE_HALF_TRANSFORM = 1,  /* X = B C_act (the dominant contraction) */
  DONOF_PHASE_MO_3INDEX = 2,       /* b^P = C_act^T X^P */
  DONOF_PHASE_JK_Y = 3,            /* J, K accumulation and the Y^P operands */
  DONOF_PHASE_G_BUILD = 4,         /* G += sum_P X^P Y^P */
  DONOF_PHASE_ENERGY_LAMBDA = 5,   /* E, dE/dgamma, lambda = C^T G */
  DONOF_PHASE_BACKWARD = 6,        /* donof_energy_backward */
  DONOF_PHASE_PREPARE_B = 7,       /* donof_prepare_B */
  DONOF_PHASE_ORBITAL_UPDATE = 8,  /* donof_orbital_update */
  DONOF_PHASE_OCC_OPT = 9,         /* donof_optimize_occupations */
  DONOF_PHASE_ORBITAL_STEP = 10,   /* one diagonalisation step of donof_optimize */
  DONOF_NUM_PHASES = 11
};
int donof_profile_enable(int32_t enable);
int donof_profile_read(int32_t phase, double* total_ms, int32_t* intervals);
int64_t donof_launch_count(void);

/* Human-readable text for a status code (static storage). */
const char* donof_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* DONOF_H */
