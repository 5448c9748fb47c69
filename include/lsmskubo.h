/*
 * lsmskubo.h -- C ABI of the GB300 (sm_103a) LSMS Kubo-Greenwood conductivity
 * library (arXiv 2311.12134).
 *
 * The library computes, for every atom m of a supercell, the local interaction
 * zone (LIZ) KKR matrix M = T^{-1} - g at complex energies z, its LU factors,
 * the central scattering-path blocks tau^{n0} (Eq. tau-inverse restricted to the
 * LIZ, Sec. II.A and Fig. 1), the LSMS Kubo-Greenwood traces
 * (Eq. lsms-conductivity-formula), their four-combination consolidation into
 * sigma (Eq. sigma-tilde-consolidation) and rho = sigma^{-1} (end of Sec. II.B),
 * plus the gradient of sigma with respect to the per-site inverse t-matrices.
 *
 * Conventions (readings of the paper, which fixes none of them):
 *  - Rydberg atomic units (hbar = 1, m_e = 1/2): kappa = sqrt(z) (principal
 *    root) and the prefactor 4 m_e^2 / hbar^3 of Eq. (lsms-conductivity-formula)
 *    is 1; N Omega is the supercell volume; no spin factor.
 *  - Real spherical harmonics without the Condon-Shortley phase; channel index
 *    L = l*l + l + m; K = (lmax+1)^2 channels per site; lmax in 0..3.
 *  - g^{nm}_{LL'}(z) = -4 pi i kappa sum_L'' i^{l-l'-l''} C_{LL'L''} h1_{l''}(kappa R) Y_L''(R^)
 *    with R = R_m - R_n (row site n, column site m) for Im z >= 0, and the
 *    decaying (advanced) form +4 pi i kappa sum ... h2_{l''}(kappa R) ... for
 *    Im z < 0, so g(z*) = conj g(z).  On-site blocks of g are zero.
 *  - Energies come in pairs per broadening delta: z[2d] = E_F + i delta_d,
 *    z[2d+1] = E_F - i delta_d.
 *  - Current matrices J are indexed by the energy pair (z_a, z_b):
 *    c = 0 (+,+), 1 (+,-), 2 (-,+), 3 (-,-); in the term of combination
 *    c = (z1, z2), site m carries J(z2, z1) and site n carries J(z1, z2).
 *  - t^{-1} blocks must be complex-symmetric (true for scatterers with time
 *    reversal symmetry in a real-harmonic basis).  Then M^T = M and the row block
 *    is tau^{0n} = (tau^{n0})^T, which the library uses.  The assembly checks it:
 *    a block with max |t - t^T| > 1e-12 max |t| (|.| = |Re| + |Im|) flags every
 *    unit whose LIZ holds that site LSMS_UNIT_TINV_ASYM, and those units' results
 *    are not valid.
 *
 * Memory: "dev" = device pointer on the current CUDA device, "host" = host
 * pointer.  The caller owns every buffer it passes; the library owns only the
 * lsms_liz object (host arrays plus device copies made on first use on a
 * device).  Complex numbers are lsms_complex = two doubles (re, im), i.e. the
 * layout of numpy/torch complex128.  Matrices are row-major unless stated.
 *
 * Calls that take a stream enqueue work on it and return without waiting;
 * errors found on the host are returned at once.  Per-unit numerical status is
 * written to device arrays.  The library never aborts and has no CPU fallback:
 * every step of the computation runs in its CUDA kernels.
 *
 * Graph capture: the first compute call with a given lsms_liz on a device
 * uploads tables and builds the work plan (synchronous); later calls with the
 * same sizes allocate nothing when a workspace is passed, so they can be
 * captured into a CUDA graph.
 *
 * Concurrency inside a call: lsms_tau_blocks and lsms_kubo_sigma_backward split
 * each chunk of units at atom boundaries into up to four parts (option
 * "streams", else the environment variable LSMS_STREAMS, 1..4, read once;
 * default 4) that run on the caller's
 * stream and on side streams, forked from and joined back into the caller's
 * stream by events (a capture records them as graph edges).  The side streams
 * are created by the first such call on each host thread and device.  With the
 * kernel timers on (lsms_kernel_timer_enable) everything runs on the caller's
 * stream.  Results do not depend on the split.
 */
#ifndef LSMSKUBO_H
#define LSMSKUBO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } lsms_complex;
typedef struct lsms_liz lsms_liz;

enum lsms_status {
  LSMS_OK = 0,
  LSMS_ERR_ARG = -1,      /* bad argument; nothing was enqueued */
  LSMS_ERR_CUDA = -2,     /* a CUDA runtime call failed */
  LSMS_ERR_SINGULAR = -3, /* per-unit status: zero pivot */
  LSMS_ERR_NOCONV = -4,   /* per-unit status: refinement did not converge */
  LSMS_ERR_TIMEOUT = -5,  /* a bounded device wait gave up */
  LSMS_ERR_NOMEM = -6     /* workspace too small / allocation failed */
};

enum lsms_precision {
  LSMS_FP64 = 0,   /* plain form: complex128 LU and solves (DFMA) */
  LSMS_MIXED = 1   /* complex64 LU and solves, FP64 residual and iterative
                      refinement of the tau column block to FP64 accuracy */
};

/* Flag OR-ed into the precision argument of lsms_tau_blocks,
 * lsms_kubo_sigma_backward, lsms_tau_workspace_bytes,
 * lsms_backward_workspace_bytes and lsms_lu_store_bytes: conjugate pairs.
 * The energies come in pairs z[2d + 1] = conj z[2d] (checked on the host,
 * exactly; LSMS_ERR_ARG otherwise) whose t^{-1} blocks are conjugate too
 * (checked on the device to 1e-12 of the block's largest entry; a pair that
 * fails sets LSMS_UNIT_BAD_INPUT on the second energy's units).  Then
 * M(conj z) = conj M(z) in the real-harmonic basis (g(z*) = conj g(z)), so
 * only the first energy of each pair is assembled and factored:
 * tau(conj z) = conj tau(z), and the adjoint solves M(conj z) X = B as
 * X = conj(M(z)^{-1} conj B) with the first energy's factors.  The solves
 * and refinement of the second energies are skipped in the forward (their
 * unit_status words copy the first energy's); lu_store then holds the first
 * energies' factors only, so use the flag in both calls or in neither. */
#define LSMS_CONJ_PAIRS 0x100

/* Flag OR-ed into the precision argument of lsms_tau_workspace_bytes and
 * lsms_backward_workspace_bytes only: the sizes for a call that is given an
 * lu_store, so the factors (and the mixed form's double-float M) live there
 * and not in the workspace. */
#define LSMS_WS_STORE 0x200

/* Unit status values written to unit_status[e][m] (0 = fine).  Every flag
 * except LSMS_UNIT_FP64_FALLBACK means the unit's results are not valid. */
#define LSMS_UNIT_OK 0
#define LSMS_UNIT_ZERO_PIVOT 1
#define LSMS_UNIT_NOCONV 2
#define LSMS_UNIT_NONFINITE 4
#define LSMS_UNIT_BAD_INPUT 8   /* a species index outside 0..n_species-1 */
#define LSMS_UNIT_TINV_ASYM 16  /* a t^{-1} block of the LIZ is not complex-symmetric */
#define LSMS_UNIT_GROWTH 32     /* mixed form: pivot growth of the complex64 factors above the limit */
#define LSMS_UNIT_FP64_FALLBACK 64  /* mixed form: re-solved in the FP64 form on the GPU (valid result) */
#define LSMS_UNIT_TIMEOUT 128   /* a bounded device wait gave up (results invalid) */
/* Bits 8-15 of a status word: refinement sweeps; 16-23: convergence probes;
 * 24-30: pivot growth g = max|U| / max|M| of the complex64 factors when the
 * call factored or re-checked them (mixed form), as the code
 * floor(log2 g) + 64 clamped to 1..127 (127 also for a non-finite g); 0 = not
 * recorded.  The LSMS_DEBUG_BOUNDS build also sets LSMS_UNIT_BAD_INPUT when a
 * device-side index check fails (a pivot outside its range); the access is
 * skipped. */

/* ---------------------------------------------------------------- LIZ
 * Sec. II.A, Fig. 1: the LIZ of atom m holds every site within r_liz of it.
 * pos      host [n_atoms][3] atom positions (bohr), not wrapped.
 * lattice  host [3][3] rows a1, a2, a3 of the periodic cell (bohr), or NULL
 *          for a finite cluster (no images).
 * r_liz    LIZ radius (bohr); a site is inside iff |d| <= r_liz + 1e-8.
 * Periodic images are distinct sites; site = pos[j] + i a1 + j a2 + k a3 with
 * integer image (i, j, k).  Order within a LIZ: the centre first, then by
 * (atom j, i, j, k).  Returns LSMS_ERR_ARG for n_atoms < 1, r_liz < 0, a
 * singular lattice or an empty result, LSMS_ERR_NOMEM if the site count
 * overflows.  *out is owned by the caller and freed with lsms_liz_destroy. */
int lsms_build_liz(const double* pos, int n_atoms, const double* lattice, double r_liz,
                   lsms_liz** out);

/* Sizes of a LIZ set: atoms, total sites S_total = sum_m S_m, max/min S_m.
 * Any output pointer may be NULL. */
int lsms_liz_sizes(const lsms_liz* liz, int* n_atoms, int64_t* total_sites, int* max_sites,
                   int* min_sites);

/* Host copies of the LIZ arrays (any may be NULL):
 * offsets host [n_atoms+1], site_atom host [S_total], image host [S_total][3],
 * disp host [S_total][3] (site position minus centre position, bohr). */
int lsms_liz_export(const lsms_liz* liz, int64_t* offsets, int32_t* site_atom, int32_t* image,
                    double* disp);

void lsms_liz_destroy(lsms_liz* liz);

/* ---------------------------------------------------------------- inputs
 * Dipole current-matrix model (input helper; the paper's J are matrix elements
 * of the current operator that a single-site solver would supply):
 *   J[s][c][mu][L][L'] = r_ll[s][c][l][l'] * C_{L L' (1, m_mu)}  for |l - l'| = 1,
 * zero otherwise; mu = x, y, z <-> m = +1, -1, 0; C the real Gaunt coefficient.
 * r_ll host [n_species][4][lmax+1][lmax+1]; J host [n_species][4][3][K][K]. */
int lsms_dipole_current(int lmax, const lsms_complex* r_ll, int n_species, lsms_complex* J);

/* Real Gaunt table C[L1][L2][L3] = int Y_L1 Y_L2 Y_L3 dOmega, L1, L2 < (lmax+1)^2,
 * L3 < (2 lmax + 1)^2, from the Wigner 3j closed form.  host output. */
int lsms_gaunt_table(int lmax, double* C);

/* ---------------------------------------------------------------- tau
 * Eq. (tau-inverse) on each LIZ: for every atom m and energy e, assemble
 * M = T^{-1} - g (n = K S_m), LU-factor it with partial pivoting (largest
 * |Re| + |Im| in the column, lowest row on ties) and solve M X = E0, E0 the
 * first K columns of the identity, so X holds the column blocks tau^{p0}.
 *
 * species      dev [n_atoms] int32 species index of each atom (< n_species).
 * tinv         dev [n_species][n_energy][K][K] t^{-1}(z_e), complex-symmetric.
 * z            host [n_energy] complex energies (Im z != 0 recommended).
 * precision    LSMS_FP64 or LSMS_MIXED, optionally | LSMS_CONJ_PAIRS.  The mixed
 *              form takes LIZ matrices up to n = K S = 16,600 (LSMS_ERR_ARG beyond).
 * tau          dev [n_energy][S_total][K][K] output: tau[e][s] = tau^{s 0} of
 *              the LIZ that site s belongs to (row L, column L').
 * unit_status  dev [n_energy][n_atoms] int32 output, or NULL: bits 0-7 the
 *              LSMS_UNIT_* flags, bits 8-15 the number of refinement sweeps,
 *              bits 16-23 the number of convergence probes (mixed form; both 0
 *              for FP64).  Mixed form: a sweep adds the complex64 correction
 *              D = (LU)^-1 (B - M X) (residual in double-float, ~2^-48) to X and
 *              stops when ||D||_F <= 1e-10 ||X||_F; after each sweep a probe
 *              takes the same test on 2 random complex Gaussian combinations of the columns
 *              (y_q = X w_q: sum_q ||(LU)^-1 (B w_q - M y_q)||^2 <= 1e-20
 *              sum_q ||y_q||^2) and stops there when it passes, so X carries
 *              the correction test's error bound without a further full sweep.  LSMS_UNIT_NOCONV after 6
 *              sweeps (option "ir_max_sweeps").
 *              Mixed form, pivot growth: the assembly records max |M| and the
 *              factorization max |U| (|.| = |Re| + |Im|); a unit with
 *              max |U| > growth_limit * max |M| (option "growth_limit", default
 *              1e3) is flagged LSMS_UNIT_GROWTH.
 *              Mixed form, FP64 fallback: after all units, up to
 *              "fallback_slots" units (default 8, in the library's unit order)
 *              flagged ZERO_PIVOT, NOCONV, GROWTH or TIMEOUT are assembled,
 *              factored and solved again in the FP64 form on the GPU within the
 *              same call; their tau blocks are overwritten, those flags cleared
 *              and LSMS_UNIT_FP64_FALLBACK set.  Units beyond the slots keep
 *              their flags.
 * workspace    dev scratch of workspace_bytes (>= lsms_tau_workspace_bytes for
 *              one unit), 256-byte aligned (else LSMS_ERR_ARG); the units are
 *              processed in chunks that fit it.  NULL = the library allocates
 *              (stream-ordered) and frees it.  The sizes include the FP64
 *              fallback slots (mixed form) at the current "fallback_slots"
 *              option; change the option before sizing a workspace.
 *              With LSMS_WS_STORE in the precision argument the sizes assume
 *              an lu_store (no factors in the workspace).
 * lu_store     dev buffer of lu_store_bytes (lsms_lu_store_bytes), 256-byte
 *              aligned, that keeps the factors and pivots (mixed form: also M as
 *              double-float pairs) for lsms_kubo_sigma_backward, or NULL.
 * stream       cudaStream_t (NULL = legacy default stream).
 */
int lsms_tau_workspace_bytes(const lsms_liz* liz, int lmax, int n_energy, int precision,
                             size_t* min_bytes, size_t* all_bytes);
int lsms_lu_store_bytes(const lsms_liz* liz, int lmax, int n_energy, int precision,
                        size_t* bytes);
int lsms_tau_blocks(const lsms_liz* liz, int lmax, const int32_t* species, int n_species,
                    const lsms_complex* tinv, const lsms_complex* z, int n_energy,
                    int precision, lsms_complex* tau, int32_t* unit_status, void* workspace,
                    size_t workspace_bytes, void* lu_store, size_t lu_store_bytes,
                    void* stream);

/* ---------------------------------------------------------------- sigma
 * Eq. (lsms-conductivity-formula) and Eq. (sigma-tilde-consolidation):
 *   S_c[mu][nu] = sum_m sum_{n in LIZ_m} Tr[J^{m mu}(z2,z1) tau^{0n}(z1) J^{n nu}(z1,z2) tau^{n0}(z2)]
 *   sigma_tilde_c = -S_c / (pi V),  sigma = (1/4)(st_0 - st_1 - st_2 + st_3),
 *   rho = (Re sigma)^{-1}.
 * J            dev [n_species][4][3][K][K] (+ d * J_delta_stride elements for
 *              broadening d; stride 0 = the same J for every delta).
 * tau          dev output of lsms_tau_blocks with n_energy = 2 n_delta.
 * volume       supercell volume N Omega (bohr^3).
 * precision    LSMS_FP64: the K x K products in FP64.  LSMS_MIXED: the K x K
 *              products and the site sums in double-float arithmetic on the FP32
 *              pipes (unit roundoff about 2^-48); the last trace, the sums over
 *              atoms and sigma, rho in FP64 in both.  Optionally
 *              | LSMS_CONJ_PAIRS: tau holds conjugate pairs, tau(z[2d+1]) =
 *              conj tau(z[2d]) (as lsms_tau_blocks writes them with that flag;
 *              not checked); when the current matrices also satisfy
 *              J(-,-) = conj J(+,+) and J(-,+) = conj J(+,-) (checked on the
 *              device to 1e-12 of the largest |J|), the (-,+) and (-,-) traces
 *              are taken as the conjugates of the (+,-) and (+,+) ones instead of
 *              being computed (half the trace work); otherwise all four are
 *              computed.
 * sigma_tilde  dev [n_delta][4][3][3] output or NULL.
 * sigma        dev [n_delta][3][3] output.
 * rho          dev [n_delta][3][3] double output or NULL.
 * Reductions over atoms are in a fixed order (bitwise reproducible). */
int lsms_kubo_sigma(const lsms_liz* liz, int lmax, const int32_t* species, int n_species,
                    const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau,
                    int n_delta, double volume, int precision, lsms_complex* sigma_tilde,
                    lsms_complex* sigma, double* rho, void* stream);

/* Per-atom terms of the same sum: sigma_tilde_atoms dev [n_delta][4][n_atoms][3][3]
 * output, entry [d][c][m] = -(1/(pi V)) S_c(m), the term of centre atom m in
 * Eq. (lsms-conductivity-formula), so that sigma_tilde = sum over m (a local
 * decomposition of the LSMS conductivity by centre atom).  Other arguments as
 * for lsms_kubo_sigma.  LSMS_MIXED takes stream-ordered scratch for the
 * double-float copy of J (as lsms_kubo_sigma does). */
int lsms_kubo_sigma_atoms(const lsms_liz* liz, int lmax, const int32_t* species, int n_species,
                          const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau,
                          int n_delta, double volume, int precision, lsms_complex* sigma_tilde_atoms,
                          void* stream);

/* Same computation and arguments as lsms_kubo_sigma, for callers that cannot
 * allocate device memory during the call: code that must not trigger cudaMalloc
 * or a stream-ordered pool allocation (a serving loop under a fixed memory
 * budget, an application that owns every byte through its own allocator, code
 * that must not add allocator synchronisation between launches).  It allocates
 * nothing: its scratch (the per-atom partial traces) is a file-scope device
 * array of 16 MiB that every GPU which loads the library holds until the
 * process exits.  The paper has no counterpart; it is a deployment variant.
 *  - Requires n_delta * n_atoms * 576 bytes plus n_delta * 576 bytes plus, for
 *    LSMS_MIXED, the double-float copy of J (n_species * 12 * K * K * 16 bytes,
 *    times n_delta when J_delta_stride != 0), each rounded up to 256, to fit in
 *    16 MiB: about 29,000 atom-delta pairs; larger problems are rejected with
 *    LSMS_ERR_ARG and a message naming the limit, before anything is enqueued.
 *  - The LIZ set must already have a device copy on the current device (made
 *    by lsms_tau_blocks, which produces tau); otherwise LSMS_ERR_ARG.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 *    first call before any stream capture.  A cudaDeviceReset (or any teardown
 *    of the device's primary context) invalidates the kept address: the library
 *    must not be used across one.
 *  - All calls share the one array: calls that can overlap on the GPU (other
 *    streams, other threads) race and corrupt each other's results; order them
 *    on one stream or synchronise between them.  Each call writes every
 *    scratch element it reads, so nothing is carried over between calls. */
int lsms_kubo_sigma_noalloc(const lsms_liz* liz, int lmax, const int32_t* species, int n_species,
                            const lsms_complex* J, int64_t J_delta_stride, const lsms_complex* tau,
                            int n_delta, double volume, int precision, lsms_complex* sigma_tilde,
                            lsms_complex* sigma, double* rho, void* stream);

/* ---------------------------------------------------------------- gradient
 * Adjoint of the two calls above.  For f = sum_{d,mu,nu} conj(w[d][mu][nu]) sigma[d][mu][nu]
 * (w = grad_sigma, dev [n_delta][3][3]) it writes, for every energy e and atom i,
 *   grad_tinv[e][i] = conj( df / d t^{-1}_i(z_e) )   (K x K, row-major),
 * the PyTorch gradient of the real loss Re f with respect to a per-site t^{-1}
 * at energy z_e (all periodic images of atom i summed).  It uses
 * d tau = -tau dM tau (from Eq. tau-inverse) with one 2K-column solve per
 * (atom, energy), reusing the LU factors (and, mixed form, the double-float M
 * of the refinement residual) from lu_store when given (same precision, same
 * inputs), else recomputing them in the workspace.
 * grad_tinv    dev [n_energy][n_atoms][K][K] output.
 * grad_tinv_species  dev [n_species][n_energy][K][K] output (the same gradient
 *              summed over the atoms of each species, i.e. with respect to the
 *              tinv argument of lsms_tau_blocks), or NULL.
 * unit_status  dev [n_energy][n_atoms] int32 output of the adjoint solves (as
 *              for lsms_tau_blocks), or NULL.
 * workspace    dev scratch of workspace_bytes (>= lsms_backward_workspace_bytes
 *              minimum, 256-byte aligned, else LSMS_ERR_ARG), or NULL for a
 *              stream-ordered allocation.
 * n_energy must be even (energies in (+, -) pairs per delta). */
int lsms_backward_workspace_bytes(const lsms_liz* liz, int lmax, int n_energy, int precision,
                                  size_t* min_bytes, size_t* all_bytes);
int lsms_kubo_sigma_backward(const lsms_liz* liz, int lmax, const int32_t* species,
                             int n_species, const lsms_complex* tinv, const lsms_complex* z,
                             int n_energy, int precision, const lsms_complex* J,
                             int64_t J_delta_stride, const lsms_complex* tau, double volume,
                             const lsms_complex* grad_sigma, const void* lu_store,
                             size_t lu_store_bytes, lsms_complex* grad_tinv,
                             lsms_complex* grad_tinv_species, int32_t* unit_status,
                             void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- options
 * Process-wide options (all threads, all devices), read at each call:
 *   "growth_limit"    pivot-growth limit of the mixed form (default 1e3; > 0)
 *   "fallback_slots"  FP64 re-solves per mixed-form call (default 8; 0..4096;
 *                     0 disables the fallback); enters the workspace sizes
 *   "ir_max_sweeps"   refinement sweeps of the mixed form before
 *                     LSMS_UNIT_NOCONV (default 6; 0..64)
 *   "streams"         concurrent parts per chunk (1..4; 0 = the environment
 *                     variable LSMS_STREAMS, else 4)
 *   "residual_tc"     1 (default): the mixed form's refinement residual for 9
 *                     or more right-hand sides runs on the tensor cores (bf16
 *                     fixed-point digits, exact FP32 accumulation, about 2^-48
 *                     of |M| |X|); 0: double-float arithmetic on the FP32 pipes
 *   "solve_cols"      right-hand-side columns per CTA of the mixed form's
 *                     triangular solves above 8 columns (8, 16 or 32; 0 = 8 up to
 *                     16 columns, else 16): a tile shape the autotuner picks
 *   "solve_regs"      0 (default): 8- and 16-column solve CTAs sized for 8 CTAs
 *                     per SM (64 registers); 1: for 4 CTAs per SM (128 registers);
 *                     2: for 6 CTAs per SM (85 registers)
 *   "nvtx"            1: NVTX ranges around the stages of each call (assembly +
 *                     LU, solve + refinement, traces, adjoint right-hand sides
 *                     and site products, FP64 fallback); 0 (default): none
 *   "solve_steps"     1: the mixed form's triangular solves run as one CTA
 *                     chain of block steps per unit and column slice (shaped by
 *                     solve_cols / solve_regs); 2: as one launch per 32-row block
 *                     step over all units of a chunk, the row update spread over
 *                     many CTAs on the FP32 pipes; 3: the same with the row
 *                     updates as 3xTF32 products on the tensor cores; 0
 *                     (default): block steps when a chunk part has fewer than two
 *                     chains per SM (few, large LIZ matrices; tensor cores from 9
 *                     columns), else chains
 * LSMS_ERR_ARG for an unknown name or a value out of range. */
int lsms_set_option(const char* name, double value);
int lsms_get_option(const char* name, double* value);

/* ---------------------------------------------------------------- call statistics
 * lsms_unit_stats: the unit_status words of a call (n_words of them, device
 * memory) reduced on the device, on `stream`, into *stats (device memory,
 * 8-byte aligned, written whole; read it after the stream's work):
 *   units            words reduced
 *   flag_units[b]    words with bit b set (b = 0..7: LSMS_UNIT_ZERO_PIVOT ..
 *                    LSMS_UNIT_TIMEOUT; b = 6 counts the FP64 re-solves)
 *   invalid_units    words with a flag other than LSMS_UNIT_FP64_FALLBACK
 *   sweeps_sum/max   refinement sweeps (mixed form)
 *   probes_sum/max   convergence probes (mixed form)
 *   growth_code_max  largest pivot-growth code (bits 24-30; 0 = none recorded)
 * One CTA, no allocation; safe inside CUDA-graph capture.  LSMS_ERR_ARG for a
 * NULL stats pointer, a NULL unit_status with n_words > 0, n_words < 0 or a
 * misaligned stats pointer. */
typedef struct lsms_stats {
  int64_t units;
  int64_t flag_units[8];
  int64_t invalid_units;
  int64_t sweeps_sum, sweeps_max;
  int64_t probes_sum, probes_max;
  int64_t growth_code_max;
} lsms_stats;
int lsms_unit_stats(const int32_t* unit_status, int64_t n_words, lsms_stats* stats, void* stream);

/* ---------------------------------------------------------------- misc */
/* Message of the last error on the calling thread ("" if none). */
const char* lsms_last_error(void);
/* Library version (major * 10000 + minor * 100 + patch). */
int lsms_version(void);
/* Number of kernel launches the library has enqueued since load (all threads). */
long long lsms_launch_count(void);
/* Per-launch CUDA-event timers (profiling aid, off by default).  enable != 0
 * clears previous records and records an event pair on the launch stream around
 * every later kernel launch; 0 stops recording.  After the caller has
 * synchronized, lsms_kernel_timer_report writes one line per kernel name,
 * "name<TAB>total_ms<TAB>launches", into buf (NUL-terminated). */
int lsms_kernel_timer_enable(int enable);
int lsms_kernel_timer_report(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* LSMSKUBO_H */
