/*
 * phx -- GB300 (sm_103a) three-phonon scattering library: C ABI.
 *
 * The library computes, for a crystal described by its second- and third-order
 * interatomic force constants (IFCs), the harmonic phonons on a q-mesh, the anharmonic
 * linewidths gamma of the modes at irreducible q-points, and the RTA lattice thermal
 * conductivity.  It follows the kALDo 2.0 paper (arXiv 2602.23728): Sec. "Interatomic
 * Force Constants" (Eqs. dynmat, dynmat_reciprocal, eigenvalue_crystal), Sec. "Group
 * Velocities" (Eq. groupvel), Sec. "Phonon Populations and Heat Capacity" (Eqs. bose,
 * heatcap), Sec. "Three-Phonon Scattering" (Eqs. gamma, phi3_proj, broadening,
 * lifetime), Sec. "Computational Implementation" (min_frequency selection) and Sec.
 * "Boltzmann Transport Equation" (Eq. rta).
 *
 * Units: Angstrom, eV, amu, ps.  Frequencies f in THz (w = 2 pi f rad/ps); linewidths
 * gamma = 1/tau in 1/ps; velocities in A/ps; conductivity in W/(m K).
 *
 * Conventions shared by every call:
 *  - Every call returns a phx_status; PHX_OK is 0.  Nothing is thrown across the ABI.
 *    After an error, phx_last_error(ctx) returns a message (owned by ctx, valid until the
 *    next call on ctx).
 *  - Array arguments marked [mem] live in host memory when mem == PHX_MEM_HOST and in
 *    device memory of the context's device when mem == PHX_MEM_DEVICE.  The caller owns
 *    all of them; the library never keeps a pointer past the call.  With host memory the
 *    call copies in and out and returns after the results are in host memory; with
 *    device memory it enqueues on `stream` (a cudaStream_t, NULL = legacy default) and
 *    returns without synchronising.
 *  - Descriptor structs (phx_cell, phx_ifc2, phx_ifc3) always point to host memory.
 *  - Complex arrays are interleaved (re, im) doubles, i.e. the C99 double _Complex layout.
 *  - Eigenvectors: evec[q][i][nu] is component i (= 3*atom + alpha) of mode nu, columns
 *    orthonormal, modes sorted by ascending frequency, gauge: the largest-modulus
 *    component of each column is real and positive (first index on ties).
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef PHX_H
#define PHX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PHX_OK = 0,
    PHX_ERR_INVALID = 1,      /* bad argument (null pointer, size, index out of range, NaN) */
    PHX_ERR_CUDA = 2,         /* CUDA runtime error (message says which)                    */
    PHX_ERR_NOMEM = 3,        /* device allocation failed                                   */
    PHX_ERR_TIMEOUT = 4,      /* a bounded device wait gave up (status word set by a kernel) */
    PHX_ERR_UNSUPPORTED = 5,  /* size or option this build does not handle                  */
    PHX_ERR_NUMERIC = 6       /* eigensolver did not converge, or non-finite results         */
} phx_status;

typedef enum { PHX_MEM_HOST = 0, PHX_MEM_DEVICE = 1 } phx_mem;
typedef enum { PHX_GAUSS = 0, PHX_LORENTZ = 1 } phx_shape;
typedef enum { PHX_FP64 = 0, PHX_TF32 = 1, PHX_BF16X3 = 2 } phx_precision;

typedef struct phx_ctx phx_ctx;
typedef struct phx_fc3 phx_fc3;

/* Unit cell: lattice rows a1, a2, a3 (A), n_atoms masses (amu).  Positions are not needed
 * by any computation (IFCs carry the geometry) and may be NULL. */
typedef struct {
    double lattice[9];
    int32_t n_atoms;
    const double* masses;
    const double* positions;
} phx_cell;

/* Second-order IFCs: n_blocks 3x3 blocks Phi2(0 i alpha, R j beta) (eV/A^2).
 * idx[5*b .. 5*b+4] = (i, j, R1, R2, R3) with R in lattice-vector units; val[9*b + 3*alpha + beta]. */
typedef struct {
    int32_t n_blocks;
    const int32_t* idx;
    const double* val;
} phx_ifc2;

/* Third-order IFCs, COO, home atom in cell 0 (eV/A^3):
 * idx[9*k .. 9*k+8] = (3a+alpha, 3b+beta, 3c+gamma, R'1, R'2, R'3, R''1, R''2, R''3),
 * val[k] = Phi3(0 a alpha, R' b beta, R'' c gamma). */
typedef struct {
    int64_t nnz;
    const int32_t* idx;
    const double* val;
} phx_ifc3;

/* Energy-conservation smearing, Eq. (broadening): Gaussian exp(-x^2/s^2)/(sqrt(pi) s) or
 * Lorentzian (s/2)/(pi (x^2 + s^2/4)) in THz; terms with |x| >= window*s are dropped
 * (window 2 in the paper; any value > 0 accepted). */
typedef struct {
    int32_t shape;        /* phx_shape */
    double sigma_thz;
    double window;
} phx_broadening;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (also made current on the calling thread). */
phx_status phx_create(phx_ctx** out, int device);
void phx_destroy(phx_ctx* ctx);
const char* phx_last_error(const phx_ctx* ctx);
/* Library version string, e.g. "phx 1.0 sm_103a". */
const char* phx_version(void);

/* Per-context options (no counterpart in the paper; they select among equivalent kernels
 * or bound the device waits):
 *   PHX_OPT_CHAIN: which kernel runs the two eigenvector contractions of the tensor-core
 *     linewidth path (Eq. (phi3_proj)): 0 = automatic (the chained kernel, which keeps the
 *     intermediate X in tensor memory, for 64 < n <= 96 modes; otherwise two GEMMs with X
 *     in device memory), 1 = the chained kernel wherever it fits (n <= 96), 2 = never.  It
 *     applies to the linewidth, multi-temperature and scattering-row passes alike.
 *   PHX_OPT_PAIR: 1 (default) = the tensor-core passes evaluate each unordered partner pair
 *     {q', q'' = -(q + q')} of the q' sum of Eq. (gamma) once, with the weights of both
 *     orderings (|V3|^2 is the same for both: Eq. (phi3_proj) is symmetric in the modes), so
 *     about half of the q' are contracted; 0 = every q' of the mesh.  Results agree to
 *     rounding.  The FP64 path always sums every q'.
 *   PHX_OPT_SIDE_SMS: the fold and Fourier stages (S3, S4) of the next q' tile run on a second
 *     stream over this many SMs while the eigenvector contractions of the current tile (the
 *     chained kernel or the two GEMMs) run on the others (M double-buffered); -1 (default) =
 *     the library's choice (48 of 152 SMs for linewidths, 34 with the scattering rows, 32 for
 *     several temperatures), 0 = one stream; at most 76.
 *   PHX_OPT_VEL_FP32: 1 = phx_harmonic forms the velocity products dD/dq E (Eq. (groupvel))
 *     with FP32 products and sums (FP64 inputs and outputs: relative error ~1e-7, far below
 *     the 1e-5 bar on kappa); 0 (default) = FP64.  The eigensolve stays FP64 either way.
 *   PHX_OPT_SC_MATRIX_FREE: phx_kappa_sc's Gamma1: 0 (default) = dense when it fits in the
 *     device memory, matrix-free otherwise; 1 = always matrix-free; 2 = always dense.
 *   PHX_OPT_HARMONIC_TR: 1 (default) = phx_harmonic solves one q of every {q, -q} pair of its q
 *     list (mod G, components within 1e-9) and fills the other by time reversal: D(-q) is the
 *     complex conjugate of D(q) (Eq. (dynmat_reciprocal) with the G-periodic phase convention),
 *     so f(-q) = f(q), e(-q) = conj e(q), v(-q) = -v(q), v (x) v unchanged; a q listed twice is
 *     copied.  0 = every q is solved on its own.  Either way every output is an FP64 solution of
 *     Eqs. (eigenvalue_crystal), (groupvel); only the basis of degenerate eigenvectors can differ.
 *   PHX_OPT_WAIT_LIMIT_NS: bound of every device barrier wait of the tensor-core kernels
 *     (default 2e9 ns); a wait that runs out makes the kernel retire and the call return
 *     PHX_ERR_TIMEOUT (host-memory calls; device-memory calls leave the status to the next
 *     host-memory call on the context).
 *   PHX_OPT_STARVE: test hook; nonzero makes the tensor-core kernels' load producers issue
 *     nothing, so the first barrier wait runs out with no copy or MMA in flight.
 * Errors: PHX_ERR_INVALID for an unknown option or a value out of range. */
typedef enum {
    PHX_OPT_CHAIN = 0,
    PHX_OPT_WAIT_LIMIT_NS = 1,
    PHX_OPT_STARVE = 2,
    PHX_OPT_PAIR = 3,
    PHX_OPT_SIDE_SMS = 4,
    PHX_OPT_VEL_FP32 = 5,
    PHX_OPT_HARMONIC_TR = 6,
    PHX_OPT_SC_MATRIX_FREE = 7
} phx_option;
phx_status phx_set_option(phx_ctx* ctx, int32_t option, int64_t value);
/* The value an option has in effect: for PHX_OPT_SIDE_SMS the SM count the tensor-core path
 * uses (the default resolved), for the others the value set.  Errors: PHX_ERR_INVALID for an
 * unknown option or a null `value`. */
phx_status phx_get_option(phx_ctx* ctx, int32_t option, int64_t* value);

/* ---------------------------------------------------------------- grid (host only)
 * Irreducible set of a Gamma-centred mesh n1 x n2 x n3 (flat index (k1*n2+k2)*n3+k3)
 * under n_rot integer rotations (rot[9*r + 3*row + col], acting on reduced q) plus time
 * reversal q -> -q (always applied): Sec. "Overview of New Capabilities" (scattering on
 * the irreducible wedge, results mapped back to the full grid).  Representatives are the
 * smallest index of each orbit, listed in ascending order.
 * Outputs (host, caller-allocated, nq = n1 n2 n3 entries each): irr[0..*n_irr), full_to_irr[nq]
 * (position in irr of each point's orbit), weight[0..*n_irr) (orbit sizes).
 * Errors: PHX_ERR_INVALID if a rotation does not map the mesh onto itself. */
phx_status phx_irreducible(const int32_t mesh[3], int32_t n_rot, const int32_t* rot,
                           int32_t* irr, int32_t* n_irr, int32_t* full_to_irr, int32_t* weight);

/* ---------------------------------------------------------------- harmonic
 * Eqs. (dynmat_reciprocal), (eigenvalue_crystal), (groupvel): for nq reduced q-points
 * q_frac[3*k..3*k+2] build D(q) = sum_R Phi2 exp(-2 pi i q.R)/sqrt(m m), diagonalise it in
 * FP64 on the GPU (batched Householder reduction + QL for n <= 96, cyclic Jacobi above) and
 * return
 *   freq_thz[nq][n]     signed frequency sign(lambda) sqrt(|lambda|)/(2 pi)          [mem]
 *   evec[nq][n][n]      complex eigenvectors (layout and gauge above)                [mem]
 *   vel[nq][n][3]       Re<e|dD/dq|e>/(2w) with the analytic derivative (0 if f<=0)   [mem, may be NULL]
 *   vv[nq][n][9]        basis-invariant v(x)v: within each degenerate set S
 *                       (|df| < 1e-5 max|f|) every mode gets
 *                       (1/|S|) sum_{m,m' in S} Re(V^a_{mm'} V^b_{m'm})/(4 w^2)         [mem, may be NULL]
 * n = 3 * cell->n_atoms, 3 <= n <= 192 for any q.
 * Larger cells (192 < n <= 8192; Eq. (eigenvalue), the real-space problem of a Gamma-only or
 * disordered cell): every q must be a lattice vector (Gamma), vel and vv must be NULL, and D is
 * real symmetric; it is solved in FP64 by Householder reduction to tridiagonal form, Sturm
 * bisection, inverse iteration (eigenvalues closer than 1e-7 ||D|| orthogonalised as a
 * cluster) and back-transformation.  evec then holds real columns (imaginary parts 0), largest
 * component positive.  Device workspace ~57 n^2 bytes (513 MB at n = 3000).
 * Errors: PHX_ERR_INVALID (block index out of range), PHX_ERR_UNSUPPORTED (q != Gamma or
 * velocities requested for n > 192), PHX_ERR_NUMERIC (no convergence / non-finite result). */
phx_status phx_harmonic(phx_ctx* ctx, const phx_cell* cell, const phx_ifc2* fc2,
                        const double* q_frac, int32_t nq,
                        double* freq_thz, double* evec, double* vel, double* vv,
                        int32_t mem, void* stream);

/* ---------------------------------------------------------------- scattering
 * Prepare the third-order IFCs for a mesh (host-side sort of the COO by lattice difference
 * d = R' - R'' folded into the mesh, upload).  The handle is immutable and may be used by
 * any number of phx_gamma calls on the same context.  Errors: PHX_ERR_INVALID for an
 * out-of-range component index. */
phx_status phx_fc3_create(phx_ctx* ctx, const phx_cell* cell, const phx_ifc3* fc3,
                          const int32_t mesh[3], phx_fc3** out);
void phx_fc3_destroy(phx_fc3* h);
int32_t phx_fc3_num_d(const phx_fc3* h);  /* number of distinct folded lattice differences */

/* Eqs. (gamma), (phi3_proj), (broadening), (lifetime) for every band of the n_irr mesh
 * points irr_q (flat mesh indices):
 *   gamma_lambda = pi hbar/(8 N_q) sum_{q' nu' nu''} |Phi(lambda, q'nu', q''nu'')|^2 / (w w' w'')
 *                  * [(1+n'+n'') delta(w-w'-w'') + 2 (n'-n'') delta(w+w'-w'')],   q'' = -(q+q')
 * with delta(w) = g(f)/(2 pi), modes with f < f_min_thz given gamma 0 and partners with
 * f' or f'' < f_min_thz skipped (decay/absorption counting as read in the library notes).
 * Inputs: freq_thz[N_q][n], evec[N_q][n][n] over the full mesh [mem]; irr_q[n_irr] [mem].
 * Outputs: gamma[n_irr][n] (1/ps) [mem]; wp2[n_irr][n] (ps^4, may be NULL): the same sum
 * with |Phi|^2 -> 1 and without pi hbar/8 (weighted two-phonon phase space).
 * prec: PHX_FP64 (all FP64, CUDA cores), PHX_TF32 or PHX_BF16X3 (V3 contraction on the
 * tcgen05 tensor cores with FP32 accumulation; weights and sums in FP32/FP64).
 * Errors: PHX_ERR_INVALID (index out of range, T <= 0, sigma <= 0), PHX_ERR_UNSUPPORTED
 * (n or mesh beyond the precision's limits). */
phx_status phx_gamma(phx_ctx* ctx, const phx_fc3* fc3, const double* freq_thz,
                     const double* evec, const int32_t* irr_q, int32_t n_irr,
                     double temperature, phx_broadening br, double f_min_thz,
                     int32_t prec, double* gamma, double* wp2, int32_t mem, void* stream);

/* Several temperatures from one contraction (paper Sec. "Performance Optimization": the
 * temperature-independent |Phi|^2 and deltas are shared, only the occupations change).
 * temperatures[n_t] (host, K); gamma[n_t][n_irr][n] (1/ps) [mem]; other arguments as phx_gamma
 * (no wp2).  Tensor-core precisions evaluate up to 4 temperatures per contraction pass (more
 * are taken in groups of 4); PHX_FP64 and the Gamma-only large cell run one full evaluation
 * per temperature.  Each gamma[t] equals phx_gamma at temperatures[t] (up to FP32 summation
 * order on the tensor-core path).  Errors: as phx_gamma; PHX_ERR_INVALID for T <= 0. */
phx_status phx_gamma_multi_t(phx_ctx* ctx, const phx_fc3* fc3, const double* freq_thz,
                             const double* evec, const int32_t* irr_q, int32_t n_irr,
                             const double* temperatures, int32_t n_t, phx_broadening br,
                             double f_min_thz, int32_t prec, double* gamma, int32_t mem, void* stream);

/* Isotope / mass-variance scattering, Eq. (isotope) (Tamura):
 *   gamma_iso(q s) = pi/(2 N_q) w^2 sum_{q' s'} delta(w - w') sum_i g_i |<e_i(q s)|e_i(q' s')>|^2
 * with the per-atom overlap <e_i|e'_i> = sum_alpha conj(e[3i+alpha]) e'[3i+alpha] (the Cartesian
 * sum inside the modulus, the frame-invariant placement), delta(w) = g(f)/(2 pi) with the
 * broadening and window of phx_gamma, modes and partners below f_min_thz skipped.  The total
 * rate of the paper is gamma = gamma_anh + gamma_iso (add the two outputs).
 * Inputs: freq_thz[nq][n], evec[nq][n][n] over the full mesh (complex; nq = N_q) [mem];
 * irr_q[n_irr] [mem]; g_atom[n/3] (host): g_i = sum_iso f (dM/M)^2 per atom of the cell.
 * Output: gamma[n_irr][n] (1/ps) [mem].  FP64 on the CUDA cores; n <= 12800.
 * Errors: PHX_ERR_INVALID (bad sizes, g < 0, sigma/window/f_min <= 0, index out of range). */
phx_status phx_gamma_isotope(phx_ctx* ctx, int32_t nq, int32_t n, const double* freq_thz,
                             const double* evec, const int32_t* irr_q, int32_t n_irr,
                             const double* g_atom, phx_broadening br, double f_min_thz,
                             double* gamma, int32_t mem, void* stream);

/* Quasi-harmonic Green-Kubo conductivity of a Gamma-only cell, Eq. (qhgk):
 *   kappa_ab = 1/V sum_{mu mu'} c_{mu mu'} Re(v^a_{mu mu'} v^b_{mu' mu}) tau_{mu mu'}
 * c_{mu mu'} = (hbar w w'/T)(n - n')/(w' - w) (the average of c_mu and c_mu' of Eq. (heatcap)
 * for |f - f'| < 1e-5 f_max); v^a_{mu mu'} = <e_mu|dD/dq_a|e_mu'>/(2 sqrt(w w')) with the
 * atom-position-gauge derivative dD/dq_a = -i sum_R (x_j + R - x_i)_a Phi2(0i, Rj)/sqrt(m m);
 * tau_{mu mu'} = g/(2((w - w')^2 + g^2)), g = (gamma_mu + gamma_mu')/4 (so tau_mu mu = 1/gamma_mu).
 * Modes below f_min_thz or with gamma <= 0 are left out; V is the cell volume.
 * Inputs: cell (lattice, positions, masses), fc2 (blocks with image vectors R), freq_thz[n],
 * evec[n][n] complex with zero imaginary parts (as phx_harmonic returns at Gamma), gamma[n]
 * (1/ps, e.g. from phx_gamma_cell) [mem]; output kappa_wmk[9] (host, W/(m K)).
 * FP64: sparse G E, dense E^T (G E) on 128 x 128 upper-triangle tiles, pair sum.  Workspace
 * 7 n^2 doubles.  The call synchronises the stream.  Errors: PHX_ERR_INVALID (complex
 * eigenvectors, bad indices, T or f_min <= 0), PHX_ERR_UNSUPPORTED (n > 8192). */
phx_status phx_kappa_qhgk(phx_ctx* ctx, const phx_cell* cell, const phx_ifc2* fc2, const double* freq_thz,
                          const double* evec, const double* gamma, double temperature, double f_min_thz,
                          double kappa_wmk[9], int32_t mem, void* stream);

/* ---------------------------------------------------------------- Gamma-only large cell
 * Eq. (phi3_proj) at q = q' = q'' = 0 and Eq. (gamma) with N_q = 1 for every mode of a
 * (disordered) cell of up to 8192/3 atoms: the real-space treatment of Gamma-only and
 * amorphous systems.  fc3 must come from phx_fc3_create with mesh {1, 1, 1}; on creation its
 * COO is summed over images and symmetrised over the permutations of (i, j, k) (a third
 * derivative is symmetric; input that already is stays unchanged).
 *   freq_thz[n] ascending or not, evec[n][n] complex with zero imaginary parts (columns are
 *   modes; as phx_harmonic returns at Gamma) [mem]; gamma[n] (1/ps) [mem].
 * The result equals the per-mode sum of phx_gamma (window, f_min and occupations alike).
 * Each unordered triple of modes is evaluated once: sparse F.e_a and W_a E on the CUDA cores,
 * E^T (W_a E) on the tensor cores (PHX_TF32, PHX_BF16X3) or FP64 CUDA cores (PHX_FP64), only
 * over 128 x 128 tiles of (b, c) that can hold a triple inside the broadening window, with the
 * three linewidth updates fused into the GEMM epilogue.  The call synchronises the stream once
 * (the frequencies plan the tiles on the host); workspace grows to ~6 GB.
 * phx_gamma with a 1x1x1-mesh handle, n > 192, n_irr = 1 and irr_q = {0} calls this.
 * Errors: PHX_ERR_INVALID (handle not 1x1x1, complex eigenvectors, bad T/sigma/f_min),
 * PHX_ERR_UNSUPPORTED (neighbour count beyond shared memory), PHX_ERR_TIMEOUT (a tensor-core
 * pipeline wait gave up; the result is then invalid). */
phx_status phx_gamma_cell(phx_ctx* ctx, const phx_fc3* fc3, const double* freq_thz, const double* evec,
                          double temperature, phx_broadening br, double f_min_thz, int32_t prec,
                          double* gamma, int32_t mem, void* stream);

/* ---------------------------------------------------------------- batched scattering
 * Many crystals (of any size up to 192 modes and any mesh) in one call: every job's
 * linewidths (as phx_gamma) and, when vv is given, its unfolded linewidths and RTA
 * conductivity (as phx_unfold + phx_kappa_rta) are enqueued as one CUDA graph, captured on the
 * first call and replayed by later calls with the same job list (same pointers and
 * parameters).  Job arrays are device memory except irr_q (host).  Precision PHX_BF16X3 or
 * PHX_TF32.  The q' tile, the contraction kernel and the side-stream share of each job class
 * (modes, mesh, lattice differences) are taken from tune[j] when tune is given and
 * tune[j].q_tile > 0; otherwise they are chosen by timing on up to three irreducible q-points
 * of the first job of the class (best of two runs each): every q' tile 8..128 with, where it fits
 * for the class, the chained kernel and the two GEMMs, at the context's side-stream share;
 * then, for the fastest (tile, kernel) and unless PHX_OPT_SIDE_SMS is set, side streams of
 * 0, 24, 32, 40, 48 and 56 of 152 SMs (scaled to the device).  Choices are cached per
 * context, and written back into tune[j] (when tune is given) for every job whose q_tile was
 * 0 on entry.
 * The call enqueues on `stream` (ordered after work already on it) and returns without
 * synchronising.  Errors: as phx_gamma; PHX_ERR_UNSUPPORTED for PHX_FP64. */
typedef struct {
    const phx_fc3* fc3;            /* prepared Phi3 of this crystal and mesh              */
    const double* freq_thz;        /* [nq][n] device                                      */
    const double* evec;            /* [nq][n][n] complex, device                          */
    const int32_t* irr_q;          /* [n_irr] host: irreducible mesh indices              */
    int32_t n_irr;
    double temperature;
    phx_broadening br;
    double f_min_thz;
    double* gamma;                 /* [n_irr][n] device, output (1/ps)                    */
    const int32_t* irr_q_dev;      /* [n_irr] device copy of irr_q (conductivity only)    */
    const int32_t* full_to_irr;    /* [nq] device (conductivity only)                     */
    const double* vv;              /* [nq][n][9] device; NULL: no conductivity            */
    double* gamma_full;            /* [nq][n] device, output (conductivity only)          */
    double volume;                 /* unit-cell volume in A^3 (conductivity only)         */
    double* kappa;                 /* [9] device, output W/(m K) (conductivity only)      */
} phx_job;

typedef struct {
    int32_t q_tile;                /* q' per Fourier tile; 0 = autotune (all three fields,
                                      written back on return)                             */
    int32_t chain;                 /* with q_tile > 0: 1 chained kernel (if it fits), 0 the
                                      two GEMMs, -1 as PHX_OPT_CHAIN                       */
    int32_t side_sms;              /* with q_tile > 0: SMs of the fold/Fourier side stream
                                      (0 = one stream), -1 as PHX_OPT_SIDE_SMS             */
} phx_tune;

phx_status phx_gamma_batched(phx_ctx* ctx, int32_t n_jobs, const phx_job* jobs, int32_t prec,
                             phx_tune* tune, void* stream);

/* ---------------------------------------------------------------- learned linewidths
 * No counterpart in the paper's equations: a small MLP ensemble that predicts log(gamma) on a
 * dense mesh from per-mode descriptors, trained on exact linewidths of a coarse subgrid by the
 * library's own forward/backward/Adam kernels (FP32).  All arrays are device memory.
 *
 * phx_features: descriptors of every band of the irreducible q-points irr_q[n_irr] of a mesh:
 *   features[s][nu][4] = (w in rad/ps, |v| in A/ps, WP2 in ps^4, n_B), where WP2 is the sum of
 *   Eq. (gamma) with |Phi|^2 -> 1 and without pi hbar/8 (same weights, window and f_min as
 *   phx_gamma), over the full mesh.  freq_thz[nq][n], vel[nq][n][3] cover the full mesh.
 *   n <= 192.  Enqueued on stream. */
typedef struct phx_mlp phx_mlp;
phx_status phx_features(phx_ctx* ctx, const int32_t mesh[3], int32_t n, const double* freq_thz,
                        const double* vel, const int32_t* irr_q, int32_t n_irr, double temperature,
                        phx_broadening br, double f_min_thz, double* features, void* stream);
/* Ensemble of `ensemble` MLPs n_in -> width (x depth hidden layers, SiLU) -> 1, initialised
 * from a counter-based generator seeded by `seed` (weights U(-sqrt(6/fan_in), +), biases 0).
 * Inputs are log(max(x, 1e-12)) standardised per feature; the target is log(gamma),
 * standardised; both standardisations are fixed by phx_mlp_train. */
phx_status phx_mlp_create(phx_ctx* ctx, int32_t n_in, int32_t width, int32_t depth, int32_t ensemble,
                          uint64_t seed, phx_mlp** out);
void phx_mlp_destroy(phx_mlp* m);
int64_t phx_mlp_num_params(const phx_mlp* m);      /* per ensemble member */
/* Parameters [ensemble][n_params] (layer by layer: W [in][out] row-major, then b [out]) and the
 * standardisation [mu_x (n_in), sd_x (n_in), mu_y, sd_y], host buffers (norm may be NULL). */
phx_status phx_mlp_get_params(phx_mlp* m, float* params, float* norm);
phx_status phx_mlp_set_params(phx_mlp* m, const float* params, const float* norm);
/* Mean-squared loss of the standardised log(gamma) and its gradient for every member on one
 * batch (X [rows][n_in], y [rows] device); loss [ensemble] and grad [ensemble][n_params] host
 * (grad may be NULL).  Synchronises the stream. */
phx_status phx_mlp_loss_grad(phx_mlp* m, const double* X, const double* y, int32_t rows, double* loss,
                             float* grad, void* stream);
/* Full-batch Adam (beta 0.9/0.999, eps 1e-8) for `epochs` steps at learning rate lr; sets the
 * standardisation from this batch.  Final losses to loss[ensemble] (host, may be NULL). */
phx_status phx_mlp_train(phx_mlp* m, const double* X, const double* y, int32_t rows, int32_t epochs,
                         double lr, double* loss, void* stream);
/* As phx_mlp_train with early stopping: the last n_val rows of (X, y) are held out (not in the
 * gradient or the standardisation); their loss is evaluated every epoch and checked every
 * check_every epochs; training stops after `patience` checks in a row without a 0.1 %
 * improvement of the ensemble-mean held-out loss, or after max_epochs, and the parameters
 * of the best check are kept.  Epochs run to *epochs_run (host, may be NULL). */
phx_status phx_mlp_train_es(phx_mlp* m, const double* X, const double* y, int32_t rows, int32_t n_val,
                            int32_t max_epochs, double lr, int32_t check_every, int32_t patience, double* loss,
                            int32_t* epochs_run, void* stream);
/* Ensemble mean and standard deviation of log(gamma) per row (device; stdv may be NULL). */
phx_status phx_mlp_predict(phx_mlp* m, const double* X, int32_t rows, double* mean, double* stdv,
                           void* stream);
/* Domain of the network: outside[r] = 1 when some input of row r (log scale, as the network
 * reads it) lies outside the range of the rows the ensemble was last trained on (the gradient
 * rows of phx_mlp_train / phx_mlp_train_es), else 0; before any training every row is inside.
 * A prediction there is an extrapolation, which the ensemble spread does not bound.
 * X [rows][n_in] and outside [rows] device arrays; enqueued on stream. */
phx_status phx_mlp_outside(phx_mlp* m, const double* X, int32_t rows, int32_t* outside, void* stream);
/* Linewidths from a prediction, for rows grouped by irreducible q-point (n_groups groups of n
 * rows, row = group * n + band): gamma[r] = exp(mean[r]) * wp2[r] (wp2 NULL: factor 1) where
 * freq_thz[r] >= f_min_thz, else 0; score[g] (optional, needs stdv) = the largest stdv over
 * the live rows of group g (0 if none), or +infinity when outside (optional, from
 * phx_mlp_outside) flags a live row of the group: the measure that picks the q-points sent
 * back to the exact kernel.  Device arrays; enqueued on stream. */
phx_status phx_mlp_reconstruct(phx_ctx* ctx, int32_t n_groups, int32_t n, const double* mean, const double* stdv,
                               const double* wp2, const double* freq_thz, double f_min_thz, const int32_t* outside,
                               double* gamma, double* score, void* stream);

/* ---------------------------------------------------------------- transport
 * Map irreducible linewidths to the full mesh (Sec. "Overview of New Capabilities"):
 * gamma_full[k][nu] = gamma_irr[full_to_irr[k]][nu] after averaging gamma_irr over each
 * degenerate set (|df| < 1e-5 max|f|) of its own q point irr_q[s], whose frequencies are
 * read from freq_full[nq][n].  [mem] for all arrays (irr_q[n_irr], full_to_irr[nq]).
 * Errors: PHX_ERR_INVALID for an index out of range (checked on host memory only). */
phx_status phx_unfold(phx_ctx* ctx, int32_t n_irr, int32_t nq, int32_t n,
                      const double* freq_full, const int32_t* irr_q, const double* gamma_irr,
                      const int32_t* full_to_irr, double* gamma_full, int32_t mem, void* stream);

/* Eq. (rta): kappa_ab = 1/(N_q V) sum_{q nu: f >= f_min, gamma > 0} c v_a v_b / gamma, with
 * c from Eq. (heatcap) (is_classic: k_B).  Velocity products from vv[nq][n][9] if vv is
 * not NULL, else from vel[nq][n][3].  kappa_wmk[9] is always host memory; the call
 * synchronises `stream`.  [mem] for freq, vel/vv, gamma_full. */
phx_status phx_kappa_rta(phx_ctx* ctx, const phx_cell* cell, int32_t nq, int32_t n,
                         const double* freq_thz, const double* vel, const double* vv,
                         const double* gamma_full, double temperature, double f_min_thz,
                         int32_t is_classic, double* kappa_wmk, int32_t mem, void* stream);

/* ---------------------------------------------------------------- iterative BTE
 * Sec. "Boltzmann Transport Equation", Eqs. (gamma1), (invBTE), (kappa_general), (sc_iter):
 * the linearised BTE for the mean free paths lambda (A, a 3-vector per mode),
 *     v_mu = Gamma0_mu lambda_mu + sum_mu' Gamma1[mu][mu'] lambda_mu',
 * solved by iteration from the RTA start lambda^(0) = v / Gamma0 (Eq. rta), with
 * kappa^(k) = 1/(N_q V) sum_mu c_mu v_mu (x) lambda^(k)_mu (quantum c, Eq. heatcap).
 *  - Unknowns: every band of the time-reversal representatives of the fc3 handle's mesh
 *    (each orbit {q, -q} keeps its smallest index; ascending, i.e. the irr list of
 *    phx_irreducible with no rotation besides the identity).  Row r = s * n + nu of
 *    representative s; R = n_tr * n rows.  lambda(-q) = -lambda(q), so points with
 *    q = -q mod G carry lambda = 0, and modes with f < f_min or Gamma0 = 0 do too.
 *  - One contraction pass in precision prec (as phx_gamma) gives Gamma0 (the linewidth
 *    gamma, 1/ps) and the off-diagonal Gamma1 (1/ps), read from Eq. (gamma1) as the
 *    linearised three-phonon collision operator: every element (q', nu', nu'') of mu's
 *    linewidth sum, with weight w (decay + absorption term), adds w f'/f at column (q', nu')
 *    and w f''/f at column (q'' = -q-q', nu''); a column of a point listed through -q is
 *    added with sign -1.  Gamma1 stays on the device, R x R in FP64 (prec = PHX_FP64) or
 *    FP32 (tensor-core precisions), when it fits in the device memory free at the call less
 *    32 GB (kept for the contraction's workspace; R x R x 4 bytes: 111 GB for 192 modes on a
 *    12^3 mesh).  Its entries are accumulated with atomic adds (FP64 or FP32), so two calls
 *    on the same inputs agree to rounding, not bit for bit.
 *  - Matrix-free form (tensor-core precisions; PHX_OPT_SC_MATRIX_FREE): when Gamma1 does not
 *    fit, or the option asks for it, nothing of order R^2 is stored: the first contraction
 *    pass gives Gamma0, and every iteration runs one more pass whose epilogue applies the same
 *    Gamma1 entries to lambda^(k) (y = Gamma1 lambda^(k), FP32 products, FP64 sums).  Each
 *    iteration then costs a contraction pass instead of a pass over Gamma1; the iterates
 *    agree with the dense form to rounding.  The FP64 path and the gamma1 output need the
 *    dense form (PHX_ERR_UNSUPPORTED / PHX_ERR_INVALID).
 *  - Iteration (Eq. sc_iter) lambda^(k+1) = (v - Gamma1 lambda^(k)) / Gamma0 stops at the
 *    first k >= 1 with |Tr kappa^(k) - Tr kappa^(k-1)| < tol |Tr kappa^(k-1)| (*converged =
 *    1), or after max_iter iterations (*converged = 0).
 * Arguments: freq_thz[nq][n], evec[nq][n][n] complex, vel[nq][n][3] (A/ps) cover the mesh
 * [mem]; temperature, br, f_min_thz, prec as phx_gamma; max_iter >= 0; tol >= 0.
 * Outputs (host): kappa_hist[(max_iter + 1) * 9] (W/(m K)), iterate k in entries 9k..9k+8
 * (row-major 3x3), k = 0 .. *n_iter; *n_iter; *converged (may be NULL).  Optional [mem]
 * outputs (NULL skips): gamma0[R], mfp[R][3] (the last iterate), gamma1[R][R] (doubles).
 * The call synchronises `stream`.  Errors: PHX_ERR_INVALID (bad argument), PHX_ERR_UNSUPPORTED
 * (a 1x1x1 mesh; too large), PHX_ERR_NOMEM, PHX_ERR_NUMERIC (a non-finite iterate: the
 * iteration diverged), PHX_ERR_TIMEOUT (a bounded device wait gave up). */
phx_status phx_kappa_sc(phx_ctx* ctx, const phx_cell* cell, const phx_fc3* fc3, const double* freq_thz,
                        const double* evec, const double* vel, double temperature, phx_broadening br,
                        double f_min_thz, int32_t prec, int32_t max_iter, double tol, double* kappa_hist,
                        int32_t* n_iter, int32_t* converged, double* gamma0, double* mfp, double* gamma1,
                        int32_t mem, void* stream);

/* ---------------------------------------------------------------- allocation-free conductivity
 * The paper has no counterpart to this call: it exists for callers that cannot allocate
 * device memory at the time they call (a host framework whose allocator owns nearly all of
 * the GPU's memory, or a time-critical loop where cudaMalloc/cudaFree, which can
 * synchronise the device, are not allowed).  It computes the same Eq. (rta) tensor as
 * phx_kappa_rta, needs no context and allocates nothing: its only scratch is a static
 * device array of 2048 x 9 doubles (144 KiB) that every GPU loading the library keeps
 * until the process exits.
 *  - All arrays are device memory of the current device: freq_thz[nq][n], vv[nq][n][9]
 *    (or vel[nq][n][3] when vv is NULL), gamma_full[nq][n]; the result goes to
 *    kappa_dev[9] (device memory, W/(m K)).  The call enqueues two kernels on `stream` and
 *    does not synchronise.
 *  - nq * n may not exceed 2048 * 2048 = 4,194,304 modes: larger inputs return
 *    PHX_ERR_UNSUPPORTED.  Bad arguments return PHX_ERR_INVALID, a failed launch or
 *    symbol lookup PHX_ERR_CUDA.
 *  - The first call on a device looks the array's address up (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.
 *  - Every call on a device shares the array and leaves its contents behind; calls that
 *    overlap on the GPU (other streams, other host threads) race on it. */
phx_status phx_kappa_rta_noalloc(const phx_cell* cell, int32_t nq, int32_t n, const double* freq_thz,
                                 const double* vel, const double* vv, const double* gamma_full,
                                 double temperature, double f_min_thz, int32_t is_classic,
                                 double* kappa_dev, void* stream);

/* ---------------------------------------------------------------- profiling
 * Kernel classes timed when profiling is on (CUDA events recorded on the launching stream
 * immediately before and after every launch of the class). */
typedef enum {
    PHX_K_DFT = 0,          /* tensor-core GEMM over lattice differences (S4)              */
    PHX_K_GEMM_E2 = 1,      /* tensor-core GEMM with e_q'' (first eigenvector contraction) */
    PHX_K_GEMM_E1 = 2,      /* tensor-core GEMM with e_q' + fused weights and reduction    */
    PHX_K_FOLD = 3,         /* Phi3 fold into the lattice-difference operand (S3)          */
    PHX_K_FP64_GEMM = 4,    /* FP64 complex GEMMs of the FP64 path                          */
    PHX_K_FP64_EPI = 5,     /* FP64 weight/reduction kernel                                 */
    PHX_K_EIGEN = 6,        /* eigensolvers (batched Householder + QL or Jacobi)            */
    PHX_K_CELL_SPARSE = 7,  /* Gamma-only cell: W_a = F e_a and X_a = W_a E (CUDA cores)      */
    PHX_K_CELL_TRANSPOSE = 8, /* Gamma-only cell: operand layout transposes                   */
    PHX_K_CELL_GEMM = 9,    /* Gamma-only cell: E^T X_a tiles + fused role-weight epilogue   */
    PHX_K_EIG_TRIDIAG = 10, /* large-cell eigensolver: dynamical matrix + Householder steps  */
    PHX_K_EIG_VECTORS = 11, /* large-cell eigensolver: inverse iteration                    */
    PHX_K_EIG_BACK = 12,    /* large-cell eigensolver: back-transformation + output          */
    PHX_K_EIG_BISECT = 13,  /* large-cell eigensolver: Sturm multisection (eigenvalues)      */
    PHX_K_SC_STEP = 14,     /* iterative BTE: one Gamma1 x mean-free-path pass (HBM-bound)   */
    PHX_K_CHAIN = 15,       /* chained e_q'' and e_q' contractions + fused weights (one kernel) */
    PHX_K_COUNT = 16
} phx_kernel_class;

/* Turn profiling on (1) or off (0); turning it on clears the counters.  Off by default. */
phx_status phx_profile_enable(phx_ctx* ctx, int32_t on);
/* Totals since the last enable for one kernel class: summed event time (ms), launches,
 * algorithmic flops (useful complex products x 8, padding excluded) and algorithmic bytes.
 * Synchronises on the recorded events.  kernel = -1 returns in *launches the number of
 * kernels of any kind this context launched since the last enable (times not summed). */
phx_status phx_profile_read(phx_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches,
                            double* flops, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* PHX_H */
