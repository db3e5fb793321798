/*
 * iscsi.h -- C ABI of the GB300 (sm_103a) Integral-Screened CI sigma library.
 *
 * The library computes sigma = H_tau c for the spin-restricted, non-relativistic
 * Hamiltonian in its index-restricted form (Sorensen, Bauch & Madsen,
 * arXiv:1609.07757, Eq. index_re), restricted to the determinants of a
 * truncated CI expansion (Eq. ci_hierarchy), where every integral term whose
 * "unit" has magnitude <= tau is dropped (integral screening, Eqs. sigma_int
 * and sigma_split; the screen sits on each integral, as in the screened loops
 * of Sec. "Second part").  The units are
 *   one-body       h_pq                       (operators a+_p a_q, either spin)
 *   same-spin      g_psrq - g_pqrs, p>r, q>s  (a+_p a+_r a_q a_s, either spin)
 *   opposite-spin  g_pqrs                     (-a+_pa a+_rb a_qa a_sb)
 * with g_pqrs = (pq|rs) in chemist notation.  They are grouped into the 42
 * classes of Eqs. class_to_ex_dx .. the_end (class ids below).  It also finds
 * the lowest eigenpairs of H_tau with a Davidson solver (Eq. hcec; the paper
 * names Davidson as the usual companion of the sigma step, Eq. sigma).
 *
 * Conventions
 *   - orbitals 0..n_sigma-1 are occupied in the reference determinant of spin
 *     sigma (O), the others virtual (V); the excitation level of a string is
 *     its number of electrons in V;
 *   - strings are sorted by (excitation level, colex rank sum_i C(o_i, i+1) of
 *     the ascending orbital list o_0 < o_1 < ...);
 *   - a determinant (A, B) is in the space iff level(A) + level(B) <=
 *     max_excitation; its index is off[A] + B, where B runs over the beta
 *     strings of level <= max_excitation - level(A) (a prefix of the sorted
 *     list) -- alpha-major, the CI-vector blocking of Fig. cisdt;
 *   - |A,B> = prod_{p in A ascending} a+_pa prod_{q in B ascending} a+_qb |vac>;
 *   - a context created with iscsi_init_gas counts levels against its own
 *     inner orbitals instead of the reference's (Sec. "Generalized Active
 *     Space"), with the same sorting and blocking; the class ids keep the
 *     reference's O / V.
 *
 * Beyond sigma and the Davidson solver: spin-resolved one- and two-body
 * (transition) density matrices (iscsi_density), time propagation under a
 * time-dependent one-body term (iscsi_propagate), GAS restrictions
 * (iscsi_init_gas, iscsi_set_gas), and many independent contexts at once
 * (iscsi_batch_sigma, iscsi_batch_davidson).
 *
 * Class ids (bit i of a class mask):
 *   0..3   H^{1,1}, H^{1,0}, H^{0,1}, H^{0,0} _{1,0,1}   (one-body alpha)
 *   4..7   the same for _{1,0,-1}                         (one-body beta)
 *   8..23  the 16 opposite-spin terms of H_{2,0,0}, in the order
 *          H^{2,2}, H^{2,1} (2 terms), H^{1,2} (2), H^{2,0}, H^{1,1} (4),
 *          H^{0,2}, H^{1,0} (2), H^{0,1} (2), H^{0,0}, each term's order
 *          being the paper's
 *   24..32 H^{P,H}_{2,0,2} (alpha-alpha), (P,H) = (2,2),(2,1),(1,2),(2,0),
 *          (1,1),(0,2),(1,0),(0,1),(0,0)
 *   33..41 H^{P,H}_{2,0,-2} (beta-beta), same order
 * P counts de-excitation annihilators (index in V), H de-excitation creators
 * (index in O).
 *
 * Memory and threading
 *   - one process, one GPU (the device current at iscsi_init); calls are not
 *     thread-safe;
 *   - "device" pointers must point to memory of that GPU, 8-byte aligned;
 *   - every call returns after enqueueing its work on the library stream
 *     (iscsi_set_stream) unless stated otherwise;
 *   - the library owns the device memory it allocates; the caller owns every
 *     buffer it passes in, and the library never keeps a pointer to it after
 *     the call returns.
 */
#ifndef ISCSI_H
#define ISCSI_H

#if defined(__GNUC__)
#define ISCSI_API __attribute__((visibility("default")))
#else
#define ISCSI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int iscsi_status;

#define ISCSI_OK 0
#define ISCSI_E_ARG (-1)      /* invalid argument                                  */
#define ISCSI_E_NOMEM (-2)    /* device or host allocation failed                  */
#define ISCSI_E_CUDA (-3)     /* a CUDA call failed (see iscsi_last_error)          */
#define ISCSI_E_NOCONV (-4)   /* Davidson hit its iteration limit; best estimates  */
#define ISCSI_E_NOINIT (-5)   /* no current context                                */
#define ISCSI_E_NAN (-6)      /* NaN or Inf detected                               */
#define ISCSI_E_WAIT (-7)     /* a bounded device wait ran out                     */

/* Limits: 1 <= norb <= 256; 0 <= nalpha, nbeta <= min(norb, 16); the dense
   same-spin string Hamiltonian of each spin, C(norb, n_sigma)^2 doubles, must
   fit in device memory; max_excitation >= 0 (values above the largest
   possible level give full CI). */

/*
 * Create a context for n = norb orbitals, nalpha / nbeta electrons, CI space
 * truncated at total excitation level max_excitation (Eq. ci_hierarchy), and
 * make it current.
 *   h1   host, n*n doubles, row-major h_pq: the one-body part
 *        sum_pq h_pq (a+_p a_q) of each spin.  Any real matrix: the
 *        Hamiltonian's (symmetric), or a general one-body operator such as
 *        a transition operator a+_p a_q (h = e_p e_q^T, not symmetric); the
 *        eigen-solvers and the propagator need a symmetric h1 (ISCSI_E_ARG
 *        otherwise), sigma and the counts take any.
 *   eri  host, npair*npair doubles, npair = n(n+1)/2, pair-packed chemist
 *        integrals: (pq|rs) = eri[P(p,q)*npair + P(r,s)] with
 *        P(p,q) = max(p,q)*(max(p,q)+1)/2 + min(p,q).  The matrix must be
 *        symmetric ((pq|rs) = (rs|pq)); eri may be NULL (no two-electron part).
 *        The two-body part is (1/2) sum (pq|rs) (E_pq E_rs - delta_qr E_ps)
 *        (Eq. ham): the electron repulsion, or any two-body property
 *        operator with these symmetries (the square of a one-body operator
 *        d, say: (pq|rs) = 2 d_pq d_rs with h1 = d d).
 *   tau  screening threshold, >= 0: a unit u is kept iff |u| > tau
 *        (the algorithm's "if |I| > epsilon", Sec. "Second part").
 * The library copies h1 and eri; the caller may free them on return.  Builds
 * the string spaces, determinant addressing, screened units and work lists on
 * the device (once per context) and synchronises before returning.
 * Errors: ISCSI_E_ARG (limits above, tau < 0 or NaN, NULL h1), ISCSI_E_NOMEM,
 * ISCSI_E_CUDA.  On error no context is created and the current context is
 * unchanged.
 */
ISCSI_API iscsi_status iscsi_init(int norb, int nalpha, int nbeta, int max_excitation, const double* h1, const double* eri,
                        double tau);

/*
 * Create a context on a GAS space (Sec. "Generalized Active Space"): the
 * determinants of nalpha / nbeta electrons in norb orbitals whose accumulated
 * subspace occupations satisfy the limits (sizes, cmin, cmax as in
 * iscsi_set_gas; no excitation-level truncation beyond them), and make it
 * current.  The library computes on an enclosing truncated space and masks the
 * rest: of full CI and, for each subspace boundary j < nspace - 1, the space
 * of determinants with at most N - cmin[j] electrons (N = nalpha + nbeta)
 * outside the first sizes[0] + ... + sizes[j] orbitals (a level truncation
 * with those orbitals as the inner ones), it takes the smallest; the limits
 * it does not enforce are applied as by iscsi_set_gas.  With one lower limit
 * doing all the restricting (the paper's "at most one electron in the
 * continuum") no mask remains and sigma costs what the GAS space costs.
 * iscsi_ndet is the enclosing space's dimension; iscsi_stats gives "gas_ndet"
 * (the GAS dimension) and "level_split" (the inner orbitals per spin); strings
 * are sorted by the level of that split (electrons outside the inner orbitals),
 * determinants by it as in iscsi_init.  h1, eri, tau as in iscsi_init.
 * Errors: ISCSI_E_ARG (limits of iscsi_init and iscsi_set_gas), ISCSI_E_NOMEM,
 * ISCSI_E_CUDA.  On error no context is created.
 */
ISCSI_API iscsi_status iscsi_init_gas(int norb, int nalpha, int nbeta, int nspace, const int* sizes, const int* cmin,
                                      const int* cmax, const double* h1, const double* eri, double tau);

/*
 * sigma = H_tau c for nvec vectors (Eq. sigma, screened as Eq. sigma_split).
 *   c      device, FP64, [nvec][ndet] (vector-major, ndet contiguous).
 *   sigma  device, FP64, [nvec][ndet]; overwritten; must not overlap c.
 * Arithmetic follows the "precision" option (64: FP64 throughout; 32: FP32
 * products and accumulation, inputs rounded to FP32, result widened to FP64).
 * Asynchronous on the library stream; does not synchronise except the first
 * time a new nvec is used (work lists are uploaded once per nvec).  A bounded
 * device wait that runs out inside the tensor-core kernels is reported as
 * ISCSI_E_WAIT by the next synchronising call (iscsi_sigma_host,
 * iscsi_davidson).
 * Errors: ISCSI_E_NOINIT, ISCSI_E_ARG (NULL pointers, nvec < 1), ISCSI_E_NOMEM
 * (workspace growth), ISCSI_E_CUDA (launch failure).
 */
ISCSI_API iscsi_status iscsi_sigma(const void* c, void* sigma, int nvec);

/*
 * Allocation-free variant of iscsi_sigma: FP64, one vector, on the current
 * context.  (The paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory when they need sigma -- code
 * under a memory manager that owns all device memory, or real-time and
 * callback contexts where cudaMalloc, which may synchronise the device, is not
 * allowed.)  It allocates nothing: the lifted vector, the contraction product
 * and the GEMM problem lists live in one static 32 MiB device array that every
 * GPU loading this library holds until the process exits.  It computes on the
 * FP64 FMA kernels (the route of option fp64_tc = 0), not on the tensor
 * cores.  The problem lists stay in the array: a call copies them from host
 * memory only when the array last served another context.
 *   c      device, FP64 [ndet]; sigma: device, FP64 [ndet], overwritten.
 * The context must need at most 32 MiB of scratch (full CI with 2+2
 * electrons: up to 38 orbitals); larger contexts are rejected with
 * ISCSI_E_ARG and a message naming the bytes needed.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the array: calls
 * whose work overlaps on the GPU race and must be serialised by the caller.
 * Asynchronous on the library stream.  A context with a determinant mask
 * (iscsi_set_gas) is refused with ISCSI_E_ARG.  Errors: ISCSI_E_NOINIT,
 * ISCSI_E_ARG, ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_sigma_noalloc(const void* c, void* sigma);

/*
 * Same as iscsi_sigma with HOST buffers: copies c to the device, computes,
 * copies sigma back and synchronises.  c, sigma: host, [nvec][ndet] FP64
 * (page-locked memory gives the fastest copies).  The device staging buffers
 * (2 nvec ndet doubles) stay with the context for later calls until it is
 * destroyed.
 */
ISCSI_API iscsi_status iscsi_sigma_host(const double* c, double* sigma, int nvec);

/*
 * One- and two-body (transition) density matrices of Eqs. d1 and d2 (Sec.
 * "Density matrices"), spin-resolved, for the current context's space:
 *   d1[s][p][q]       = <bra| a+_{p s} a_{q s} |ket>,  s = 0 alpha, 1 beta;
 *   d2[b][p][q][r][t] = <bra| a+_{p s} a+_{r u} a_{t u} a_{q s} |ket>,
 *                       (s, u) = (alpha, alpha), (alpha, beta), (beta, beta)
 *                       for b = 0, 1, 2; flat index ((p n + q) n + r) n + t
 *                       inside each block.
 * The spin-summed matrices of Eqs. d1 and d2 are d1[0] + d1[1] and
 * d2[0] + d2[2] + d2[1] + d2[1] with (p,q) and (r,t) exchanged; with these
 * blocks <bra|H|ket> (tau = 0) = sum h_pq (d1[0] + d1[1])_pq
 * + 1/2 sum g_pqrt (d2[0] + d2[2])_pqrt + sum g_pqrt d2[1]_pqrt.
 *   bra  device, FP64 [ndet].
 *   ket  device, FP64 [ndet], or NULL (or bra) for the state densities of
 *        bra; then the symmetric half of the contraction is computed.
 *   d1   device, FP64 [2][n][n], or NULL;  d2: device, FP64 [3][n^4], or NULL
 *        (at least one of them); overwritten.
 * The two-body blocks are FP64-accurate products of lifted vectors on the
 * tensor cores (exact bf16 slices); the first call with d2 builds the string
 * tables and work lists and synchronises; later calls are asynchronous on the
 * library stream.  Workspace: about 14 bytes per element of the lifted
 * vectors (n^2 rows x the hole-pair count for the alpha-beta block) plus the
 * pair-indexed results (n^4 doubles); a ket different from bra adds its own
 * slices.  A bounded device wait that runs out is reported by the next
 * synchronising call.
 * Errors: ISCSI_E_NOINIT, ISCSI_E_ARG (bra NULL, both outputs NULL), ISCSI_E_NOMEM,
 * ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_density(const void* bra, const void* ket, void* d1, void* d2);

/*
 * Same as iscsi_density with HOST buffers (bra, ket [ndet]; d1 [2 n n]; d2
 * [3 n^4]): copies in, computes, copies out, synchronises and reports a
 * device wait that ran out (ISCSI_E_WAIT).  Its device staging buffers stay
 * with the context for later calls until it is destroyed.
 */
ISCSI_API iscsi_status iscsi_density_host(const double* bra, const double* ket, double* d1, double* d2);

/*
 * Time propagation of a CI vector under H(t) = H_tau + f(t) V (Eq. ham with a
 * time-dependent one-body part h(t) = h + f(t) v; the two-body part constant)
 * by the short-iterative Lanczos propagator (the paper's SIAL): per step of
 * length dt, with the field held at its sample f_k, a Krylov space of krylov
 * vectors of H_tau + f_k V from the current vector, the exponential of its
 * tridiagonal matrix, and the combination.  The basis is kept orthogonal by
 * two Gram-Schmidt passes; the small eigenproblem runs on the host.
 *   c         device, FP64, updated in place: real time [2][ndet] (real part,
 *             then imaginary part), c <- exp(-i H_k dt) c per step; imaginary
 *             time [ndet], c <- exp(-H_k dt) c / |exp(-H_k dt) c| (the paper's
 *             ground-state runs).
 *   nsteps    >= 1;  dt: finite, != 0 (> 0 in imaginary time; < 0 propagates
 *             backwards in real time).
 *   field     host [nsteps] samples f_k (for a smooth field, its value at the
 *             step's midpoint), or NULL for f = 0.
 *   coupling  handle of a context created with iscsi_init(norb, nalpha, nbeta,
 *             max_excitation, v, NULL, tau) on the same space (for a context
 *             from iscsi_init_gas: iscsi_init_gas with the same limits and v,
 *             NULL), or 0 when field is NULL.  For each step its string matrices, scaled by f_k, are
 *             added to the current context's (the one-body classes become
 *             per-step), so a Krylov vector costs one sigma; the current
 *             context is restored exactly when the call returns.
 *   krylov    Krylov dimension, 2..64 (12 is typical).
 *   imaginary 0: real time, 1: imaginary time.
 *   diag      host [2 * nsteps] or NULL: per step the error indicator
 *             |c| beta_m |e_m^T exp(.) e_1| of the Krylov approximation and
 *             <c|H_k|c> / <c|c> at the step's start.
 * Sigma runs in the "precision" option's arithmetic.  Synchronises (twice per
 * step).  Errors: ISCSI_E_NOINIT, ISCSI_E_ARG (arguments, a coupling on another
 * space, a field without a coupling, a context or coupling whose h1 is not
 * symmetric), ISCSI_E_NAN, ISCSI_E_NOMEM, ISCSI_E_CUDA, ISCSI_E_WAIT.
 */
ISCSI_API iscsi_status iscsi_propagate(void* c, int nsteps, double dt, const double* field, int coupling, int krylov,
                                       int imaginary, double* diag);

/*
 * Generalised-active-space restriction of the current context's determinant
 * space (Sec. "Generalized Active Space"; the paper's use: at most one
 * electron in a continuum subspace).  The orbitals are split into nspace
 * ordered subspaces, subspace j holding the next sizes[j] orbitals; a
 * determinant of the truncated space is kept iff for every j
 *     cmin[j] <= electrons (alpha + beta) in subspaces 0..j <= cmax[j].
 * The CI problem becomes P H_tau P, P the projector onto the kept
 * determinants, on the unchanged index range (length ndet, canonical order):
 *   iscsi_sigma, iscsi_sigma_host  sigma = P H_tau P c (zero outside);
 *   iscsi_davidson, iscsi_batch_davidson  eigenpairs of P H_tau P on the kept
 *             determinants (start vectors projected; nroots <= kept count);
 *   iscsi_propagate  c is projected first, then propagated under P H(t) P.
 * iscsi_sigma_noalloc and iscsi_batch_sigma refuse a restricted context
 * (ISCSI_E_ARG).  Density matrices and the diagonal are unaffected.  The
 * enclosing truncated space is what is computed on: the restriction selects
 * determinants, it does not make sigma cheaper.
 *   nspace    1..8, or 0 to remove the restriction (the other pointers unused).
 *   sizes     host [nspace], each >= 1, summing to norb.
 *   cmin, cmax host [nspace], 0 <= cmin[j] <= cmax[j] <= nalpha + nbeta.
 *   ndet_gas  host, out (may be NULL): the number of kept determinants (may
 *             be 0).
 * Synchronises.  The mask costs one byte per determinant of device memory.
 * Errors: ISCSI_E_NOINIT, ISCSI_E_ARG, ISCSI_E_NOMEM, ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_set_gas(int nspace, const int* sizes, const int* cmin, const int* cmax,
                                     long long* ndet_gas);

/*
 * The current context's determinant mask: mask device, uint8 [ndet], 1 for a
 * kept determinant, 0 otherwise (all 1 without a GAS restriction).
 * Asynchronous on the library stream.  Errors: ISCSI_E_NOINIT, ISCSI_E_ARG
 * (NULL), ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_gas_mask(void* mask);

/*
 * Lowest nroots eigenpairs of H_tau by a Davidson iteration on the device
 * (diagonal preconditioner, FP64 orthonormalisation, Rayleigh-Ritz and
 * residuals).  Converged when every root has residual 2-norm <= tol and its
 * energy changed by <= "etol" (option, default 1e-10) in the last iteration.
 *   energies  host, nroots doubles (output; best estimates on ISCSI_E_NOCONV).
 *   vecs      device, FP64 [nroots][ndet]: if non-NULL and option
 *             "guess_from_vecs" is 1, used as the start vectors; on return
 *             holds the (unit-norm) eigenvectors.  May be NULL.
 * With option "precision" = 32 the sigma steps run in FP32 until the residual
 * reaches "switch_tol" (option), then in FP64 for the refinement.
 * Synchronises.  Errors: ISCSI_E_NOINIT, ISCSI_E_ARG (nroots < 1 or > ndet,
 * tol <= 0, h1 not symmetric), ISCSI_E_NOCONV, ISCSI_E_NAN, ISCSI_E_NOMEM,
 * ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_davidson(int nroots, double tol, double* energies, void* vecs);

/*
 * Exercises the failure path of the tensor-core kernels' bounded waits
 * without a fault (the paper has no counterpart; this is the library's own
 * failure detection): one CTA waits, with the kernels' own bounded wait, on a
 * barrier that nothing arrives on, gives up after `polls` polls and reports
 * through the current context's error word.  The call synchronises and returns
 * ISCSI_E_WAIT with the wait's site, CTA and position in iscsi_last_error
 * ("a stage's data (MMA thread), CTA 0, position 1"), as a contraction whose
 * wait ran out would; the word is cleared and the context stays usable.
 *   polls  in [1024, 2^24] (about a microsecond per 100 polls).
 * Errors: ISCSI_E_NOINIT, ISCSI_E_ARG (polls out of range), ISCSI_E_CUDA;
 * ISCSI_E_WAIT is the expected result.
 */
ISCSI_API iscsi_status iscsi_check_bounded_wait(long long polls);

/*
 * Self-check of the host-built schedule of the persistent FP64-accurate
 * contraction (the paper has no counterpart: it is how this library spreads
 * the opposite-spin products over the SMs).  Host only: needs no context and
 * no GPU.  Plans nprob synthetic problems T_p[M_p][N_p] = sum over the
 * problem's segments of A_g B_g^T (inner dimension K_g, B_g with nrows_b_g
 * valid rows, no screened blocks) for nsm SMs and checks the plan: every
 * 128 x 64 output tile's K steps covered exactly once, split tiles' parts
 * numbered in K order on one counter and one run of workspace blocks, no CTA
 * without work.
 *   M, N, nseg  host, nprob ints each (M, N in [1, 2^24]; nseg in [1, 64]).
 *   K, nrows_b  host, sum(nseg) ints each, the segments problem by problem
 *               (K a multiple of 16 in [0, 2^24]; 1 <= nrows_b <= N).
 *   nsm         SMs to plan for, in [1, 1024].
 *   balance     host, 1 double (output): the cost model's mean CTA load over
 *               the busiest CTA's.
 *   counts      host, 5 ints (output): CTAs, work items, output tiles, split
 *               tiles, faults found (0 for a correct plan).
 * Errors: ISCSI_E_ARG (limits above, more than 2^20 tiles, NULL arrays).
 */
ISCSI_API iscsi_status iscsi_check_schedule(int nprob, const int* M, const int* N, const int* nseg, const int* K,
                                            const int* nrows_b, int nsm, double* balance, int* counts);

/* number of determinants of the current context, or -1 if none */
ISCSI_API long long iscsi_ndet(void);

/* number of strings of the given spin (0 = alpha, 1 = beta), or -1 */
ISCSI_API long long iscsi_nstrings(int spin);

/*
 * Copy the sorted strings of one spin to the host.
 *   orbitals  host, [count][n_sigma] ints, ascending orbital list per string.
 *   levels    host, [count] ints: the level the strings are sorted by -- the
 *             excitation level (electrons outside the first n_sigma orbitals),
 *             or, in a context from iscsi_init_gas, the electrons outside its
 *             inner orbitals (iscsi_stats "level_split").  Either may be NULL.
 * Synchronises.  Errors: ISCSI_E_NOINIT, ISCSI_E_ARG.
 */
ISCSI_API iscsi_status iscsi_get_strings(int spin, int* orbitals, int* levels);

/*
 * Determinant index of (alpha orbitals, beta orbitals), each an ascending host
 * list of nalpha / nbeta orbitals; -1 if outside the truncated space (for a
 * context from iscsi_init_gas: its enclosing space) or invalid, -5
 * (ISCSI_E_NOINIT) without a context.  A determinant the GAS mask excludes
 * still has an index (its sigma entries are zero).
 */
ISCSI_API long long iscsi_det_index(const int* alpha_orbitals, const int* beta_orbitals);

/*
 * Diagonal of H_tau.  diag: device, FP64 [ndet].  Asynchronous.
 */
ISCSI_API iscsi_status iscsi_diagonal(void* diag);

/* Make cudaStream_t `stream` (NULL = legacy default stream) the stream of all
   later launches of every context. */
ISCSI_API iscsi_status iscsi_set_stream(void* stream);

/*
 * Options (process-wide; "class_mask_*" take effect at the next iscsi_init):
 *   "precision"        64 (default) or 32: arithmetic of iscsi_sigma; for
 *                      iscsi_davidson 32 selects the mixed FP32/FP64 scheme
 *   "class_mask_lo"    classes 0..31 to keep, as an integer bit mask (default all)
 *   "class_mask_hi"    classes 32..41, bit i-32 (default all)
 *   "maxiter"          Davidson iteration limit (default 300)
 *   "max_subspace"     Davidson basis vectors per root; 0 (default): 12 per
 *                      root up to 96 in all, at least 4 per root
 *   "etol"             Davidson energy-change threshold (default 1e-10)
 *   "switch_tol"       mixed precision: residual at which FP64 sigma starts (default 1e-6;
 *                      the switch also happens when the FP32 residual stalls near its floor)
 *   "block_extra"      Davidson iterates the wanted roots and this many more (default 0;
 *                      convergence is judged on the wanted roots)
 *   "guess_from_vecs"  1: iscsi_davidson starts from `vecs` (default 0)
 *   "use_graph"        1 (default): one Davidson iteration is captured as a
 *                      CUDA graph on first use and replayed; 0: direct launches
 *   "olsen"            1 (default): Olsen's correction in the Davidson
 *                      preconditioner; 0: plain diagonal preconditioner
 *   "fp64_tc"          1 (default): with precision 64, the opposite-spin
 *                      contraction runs on the bf16 tensor cores with FP64
 *                      accuracy (operands cut into exact 7-bit slices, exact
 *                      integer accumulation of the leading levels; relative
 *                      error ~1e-14 of sum |g||c|); 0: native FP64 FMA
 *   "samespin_tc"      1 (default): the same for the same-spin level blocks
 *                      with more than 16 rows and 16 allowed beta strings
 *   "fp32_tc"          1 (default): with precision 32, both contractions run
 *                      on the tensor cores with three bf16 terms per element
 *                      and FP32 accumulation; 0: FP32 FMA kernels
 *   "autotune"         1 (default): before the first sigma of a context for a
 *                      given precision and vector count, time the candidate
 *                      kernel routings (opposite-spin contraction on the
 *                      tensor cores or on the FMA kernels; same-spin
 *                      level-block threshold
 *                      16/64/256/none) that a flop model puts within 3x of
 *                      the best, and keep the fastest (iscsi_stats
 *                      "route_fp64" / "route_fp32"); 0: the defaults
 *   "phase_timing"     1: record per-phase CUDA events of every sigma call
 *                      (reported by iscsi_stats; the record restarts when set)
 * Errors: ISCSI_E_ARG for an unknown key or a value out of range.
 */
ISCSI_API iscsi_status iscsi_set_option(const char* key, double value);

/*
 * Statistics of the current context as one JSON object (NUL-terminated,
 * truncated to len bytes): sizes, surviving units per group, updates per
 * sigma (one update = one sigma_I += sign * unit * c_J, counted over
 * surviving units and in-space determinant pairs), last sigma time, and of
 * the last iscsi_davidson: iterations, those of the FP32 phase, whether a
 * captured graph was replayed, time, and the largest residual norm per
 * iteration ("davidson_rmax", up to 400 values).
 * Errors: ISCSI_E_NOINIT, ISCSI_E_ARG (also when len is too small; the
 * truncated text is still written).
 */
ISCSI_API iscsi_status iscsi_stats(char* json, int len);

/* Updates per sigma per vector of the current context (see iscsi_stats), or -1. */
ISCSI_API double iscsi_updates_per_sigma(void);

/* Message of the last failing call in this process (static storage). */
ISCSI_API const char* iscsi_last_error(void);

/* Destroy every context and free all device memory the library holds. */
ISCSI_API void iscsi_finalize(void);

/*
 * Batching form: sigma_i = H_tau(context i) c_i for count independent
 * contexts (many problems of uneven size, e.g. full CI in different orbital
 * counts) in one call.  The paper treats one problem at a time; this entry
 * point has no counterpart there.  handles: host [count] distinct context
 * handles (iscsi_ctx_current); cs, sigmas: host [count] arrays of device
 * pointers, each FP64 [nvec][ndet_i] vector-major as in iscsi_sigma (the
 * caller owns them).  The precision option applies to all.  The tensor-core
 * contractions of all contexts run as one launch each; from the second call
 * with the same handles, pointers, nvec and precision the whole batch is
 * replayed from one captured CUDA graph (option "use_graph").  The FP64
 * contraction's schedule covers the whole launch and may cut a tile along K
 * at other points than a single-context call would (each part is rounded to
 * FP64 before the parts are added), so sigma_i agrees with iscsi_sigma on
 * context i to FP64 rounding, not bit for bit; calls of one batch reproduce
 * each other exactly.  Asynchronous
 * on the library stream; the current context is unchanged.  A bounded
 * device wait that runs out in a merged launch is reported by
 * iscsi_batch_check.
 * Errors: ISCSI_E_ARG (count or nvec < 1, NULL array or vector, unknown or
 * repeated handle), ISCSI_E_NOMEM, ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_batch_sigma(const int* handles, const void* const* cs, void* const* sigmas, int count,
                                         int nvec);

/* Synchronises and returns ISCSI_E_WAIT if a bounded device wait of the last
   batch's merged launches ran out, else ISCSI_OK. */
ISCSI_API iscsi_status iscsi_batch_check(void);

/*
 * Batching form of iscsi_davidson: the lowest nroots eigenpairs of count
 * independent contexts, iterated together (one Davidson iteration of every
 * unconverged context per step, their sigma steps batched as in
 * iscsi_batch_sigma, the step captured as one CUDA graph while the set of
 * unconverged contexts is unchanged).  Options as for iscsi_davidson.
 * energies: host [count][nroots]; vecs: NULL or host [count] array of device
 * pointers (each NULL or FP64 [nroots][ndet_i], written; read as start
 * vectors when "guess_from_vecs" is set); statuses: NULL or host [count],
 * each context's own status.  Synchronises.  Returns ISCSI_OK when every
 * context converged, else the first failing context's status.
 * Errors: ISCSI_E_ARG (count or nroots < 1, nroots > ndet_i, tol <= 0, NULL
 * handles or energies, unknown or repeated handle, a context whose h1 is not
 * symmetric), ISCSI_E_NOCONV,
 * ISCSI_E_NAN, ISCSI_E_WAIT, ISCSI_E_NOMEM, ISCSI_E_CUDA.
 */
ISCSI_API iscsi_status iscsi_batch_davidson(const int* handles, int count, int nroots, double tol, double* energies,
                                            void* const* vecs, int* statuses);

/*
 * Several contexts (batching).  iscsi_init creates a context and makes it
 * current; iscsi_ctx_current returns its handle (> 0), iscsi_ctx_use makes
 * another one current, iscsi_ctx_destroy frees one.
 */
ISCSI_API int iscsi_ctx_current(void);
ISCSI_API iscsi_status iscsi_ctx_use(int handle);
ISCSI_API iscsi_status iscsi_ctx_destroy(int handle);

#ifdef __cplusplus
}
#endif
#endif /* ISCSI_H */
