/*
 * pqmc.h -- C-ABI of libpqmc.so: the projective determinant-QMC sweep with a
 * Gutzwiller-projected Neel trial state, on one NVIDIA GB300 (sm_103a).
 *
 * Paper: W.-X. Chang and Z.-X. Li, "Boosting quantum Monte Carlo and
 * alleviating sign problem by Gutzwiller projection" (arXiv 2303.13403).
 *
 *  - Model: the honeycomb Hubbard model of Eq. (2); also a square t-t' lattice.
 *  - Trial state: |psi_T> = exp(-g sum_i n_i,up n_i,dn) |psi_N> of Eq. (3), with
 *    |psi_N> the ground state of the Neel mean-field Hamiltonian H_N
 *    (honeycomb Hubbard section).
 *  - Estimator: <psi_T| e^{-Theta H} O e^{-Theta H} |psi_T> / <psi_T| e^{-2 Theta H} |psi_T>
 *    (Method section), evaluated by determinant QMC.
 *  - The Gutzwiller factor is decoupled with the Ising field of Eq. (1), read
 *    in the spin channel (cosh lambda = e^{g/2}); the U term uses the same
 *    identity with g -> dtau U (cosh alpha = e^{dtau U / 2}).
 *
 * Conventions used by every entry point:
 *  - Slices tau = 0 .. Ltau+1, Ltau = round(two_theta / dtau). Slices 0 and
 *    Ltau+1 carry the Gutzwiller fields; 1..Ltau the Hubbard fields.
 *    B_tau = e^{-dtau K} e^{V(s_tau)} (interaction slices),
 *    B_tau = e^{V(s_tau)} (Gutzwiller slices).
 *  - Fields are int8 in {-1,+1}, laid out [tau][i], (Ltau+2) x N per chain
 *    ((Ltau+2) x 3N/2 bond fields for PQMC_HONEYCOMB_TV, where "site" in the
 *    Philox counter is the bond index and G has one species, spin 0).
 *  - Green's functions are G_ij = <c_i c_j^+>, row-major N x N, spin 0 = up,
 *    spin 1 = down.
 *  - One sweep is one directional pass that proposes every field once;
 *    sweeps alternate up (even sweep index) and down (odd). Measurements are
 *    taken once per sweep at tau = Ltau/2 on the freshly stabilised G.
 *  - Random numbers are Philox4x32-10 (Salmon et al., SC'11):
 *    key = (seed low, seed high word), counter = (site, slice, sweep, chain);
 *    Metropolis uniform u = ((x0 << 21) | (x1 >> 11)) * 2^-53, accept iff
 *    u < |R|; initial field s = +1 iff bit 0 of x2 is set (sweep = 0xffffffff).
 *
 * Memory and ownership: the library allocates and owns all device memory and,
 * unless a stream is supplied, its own CUDA stream on the device that is
 * current when the context is created. All pointers in these signatures are
 * HOST pointers owned by the caller; the library copies from or into them and
 * keeps no reference after the call returns.
 *
 * Errors: every entry point returns a pqmc_status; nothing is thrown across
 * the ABI and the library never aborts. After PQMC_ESTAB, PQMC_ENAN or
 * PQMC_ETIMEOUT the context keeps the error (sticky) and refuses further sweeps and
 * checkpoints until pqmc_restore loads a good checkpoint; pqmc_last_error()
 * gives a one-line reason. Entry points that read results synchronise the
 * context's stream first.
 */
#ifndef PQMC_H
#define PQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PQMC_OK = 0,
    PQMC_EINVAL = 1,    /* bad argument; nothing was changed */
    PQMC_ENOMEM = 2,    /* device or host allocation failed */
    PQMC_ECUDA = 3,     /* a CUDA call failed (launch, copy, no device) */
    PQMC_ESTAB = 4,     /* singular matrix in the stabilisation (zero pivot / zero column) */
    PQMC_ENAN = 5,      /* NaN or Inf in a ratio or in G */
    PQMC_ETIMEOUT = 6   /* a bounded device-side wait gave up: the only such wait is the
                           BF16X3 path's wait for its tensor-core products (chains kept in
                           global memory on 512-thread CTAs); every other wait is a CTA barrier */
} pqmc_status;

/* Arithmetic of the wrap and delayed-update products. The stabilisation
 * (QR, the N_sigma x N_sigma inverse of B_L B_R, log-determinant and sign)
 * is FP64 in every mode. */
typedef enum {
    PQMC_FP64 = 0,      /* everything FP64 */
    PQMC_FP32 = 1,      /* G, ratios, wrap and updates in FP32 */
    PQMC_BF16X3 = 2     /* G and ratios FP32; the wrap products as three BF16
                           tensor-core products (hi*hi + hi*lo + lo*hi), FP32
                           accumulation (tcgen05 for chains kept in global memory);
                           the rank-k delayed updates in FP32 */
} pqmc_precision;

typedef enum { PQMC_HONEYCOMB = 0, PQMC_SQUARE = 1, PQMC_HONEYCOMB_TV = 2 } pqmc_lattice_kind;

/* Lattice: honeycomb Lx x Ly unit cells (N = 2 Lx Ly; site 2(x + Lx y) + sub,
 * A(x,y) bonds to B(x,y), B(x-1,y), B(x,y-1)) or square Lx x Ly (N = Lx Ly,
 * site x + Lx y, hopping -t to nearest and -tp to next-nearest neighbours).
 * Periodic in both directions; a bond that wraps onto an existing one adds
 * its amplitude again.
 *
 * PQMC_HONEYCOMB_TV selects the spinless t-V model of the paper's second
 * model (Eq. (4)) on the same honeycomb lattice: one fermion species,
 * H = -t sum_<ij> (c^+_i c_j + h.c.) + V sum_<ij> (n_i - 1/2)(n_j - 1/2), with
 * the bond Gutzwiller trial of Eq. (5).  Its fields sit on the 3N/2 bonds
 * (bond 3 c + k of cell c = x + Lx y joins A(x,y) to B(x,y), B(x-1,y),
 * B(x,y-1) for k = 0, 1, 2), each decoupled in the density-difference
 * channel exp(kappa s (n_i - n_j)); a slice proposes its bonds class by class
 * (k = 0, 1, 2), cells ascending, and the weight is one determinant, whose
 * sign can be negative.  In its chain spec U is V, trial.g the bond
 * Gutzwiller parameter, trial.M_N the CDW field Delta_C of
 * H_C = H_0 + Delta_C sum_i eps_i n_i (raised to 1e-4 when smaller, or to
 * trial.tiebreak when that is >= 0), trial.N_up the number of fermions (< 0:
 * N/2) and trial.N_dn must be 0 or < 0. */
typedef struct {
    int kind;           /* pqmc_lattice_kind */
    int Lx, Ly;
    double t, tp;
} pqmc_lattice;

/* Trial state of Eq. (3): Gutzwiller parameter g >= 0 and the Neel field M_N
 * of H_N = H_0 + M_N sum_i eps_i (n_up - n_dn), eps_i = +1 on A, -1 on B
 * (on the square lattice (-1)^(x+y)). N_up/N_dn < 0 mean half filling.
 * tiebreak < 0 selects the default open-shell tie-break: honeycomb uses the
 * Neel field max(M_N, 1e-4); square adds tiebreak * (cos(pi x/4) + cos(pi y/2)/2)
 * on site (x, y), default tiebreak 0.2, to the trial Hamiltonian only. */
typedef struct {
    double g, M_N;
    int N_up, N_dn;
    double tiebreak;
} pqmc_trial;

/* One chain of a batch: its own lattice, couplings, projection and trial. */
typedef struct {
    pqmc_lattice lattice;
    double U, dtau, two_theta;
    pqmc_trial trial;
} pqmc_chain_spec;

typedef struct {
    int n_stab;             /* slices between QR stabilisations; Ltau/2 must be a multiple */
    int delay_k;            /* sites per delayed-update block of the Hubbard chains: 8, 16, 32
                               or 64 (accepted flips are applied to G once per block), or 0:
                               autotune (pqmc_autotune; with opts.cta_threads 0 the CTA
                               shape is tuned too).  t-V chains propose bonds in blocks of
                               16 whatever delay_k is */
    int prec;               /* pqmc_precision */
    uint64_t seed;          /* Philox key */
    int n_chains;           /* pqmc_init only: identical chains to run (>= 1) */
    int chain_offset;       /* chain index of the first chain (Philox counter word) */
    int accept_log;         /* >0: keep the accept/reject bit of the first
                               accept_log proposals per chain (test hook) */
    int max_meas;           /* capacity of per-sweep measurement records per chain (0 = 4096) */
    void* stream;           /* cudaStream_t to run on, or NULL for a library-owned stream */
    int cta_threads;        /* threads of the CTA that runs one chain: 64, 128, 256, or 512
                               (reduced paths only, one chain per SM); 0 picks 64 for FP64,
                               and for the reduced paths 256, or 512 when a chain has 128
                               sites or more. Smaller CTAs put more chains on one SM
                               (FP64: 256/cta_threads per SM, others twice that) */
    int dense_chains;       /* reduced paths only: kernels built for twice as many chains per SM
                               (fewer registers per thread); needs cta_threads 64 or 128 */
    int dg_fp64;            /* reduced paths only, diagnostic: nonzero makes the error recorded at
                               each stabilisation max |G - G_FP64|, the propagated G against
                               G_FP64 = 1 - Q_R (Q_L^T Q_R)^{-1} Q_L^T assembled in FP64 from the
                               FP64 factors (instead of against the G refreshed in the path
                               precision); 2: the G refreshed in the path precision against
                               G_FP64 (the accuracy of the refresh itself); 3: as 1, divided by
                               max(1, max |G_FP64|) per spin (the error relative to the size of
                               G). Costs two extra FP64 products per stabilisation; changes
                               nothing else (same decisions, same G) */
    int spread;             /* nonzero: sweep the chains with grid-wide kernels instead of one CTA
                               per chain, for a few large chains (one chain uses every SM): per
                               block of 32 sites a one-CTA decision kernel and a tiled update of
                               G, the wrap as tiled products, the stabilisation as tiled FP64
                               products with a blocked Cholesky QR and a blocked Gauss-Jordan
                               inverse.  Same precisions, decisions and Philox stream as the
                               one-CTA path (results agree to rounding).  Needs at most 32
                               Hubbard chains sharing N, N_sigma and Ltau; delay_k is ignored
                               (blocks of 32 sites); no dg_fp64.  PQMC_ESTAB when a stack
                               block's Cholesky factor breaks down (cond above about 1e6: use a
                               shorter n_stab) */
} pqmc_opts;

/* Sign-reweighted estimates <s O>/<s> with jackknife errors over bins of
 * consecutive sweeps (errors are NaN with fewer than two bins). E is the
 * energy per site of Eq. (2); docc the double occupancy per site; s_afm the
 * AFM structure factor of the Fig. 2 comparison, taken as its z component
 * (1/N^2) sum_ij eps_i eps_j <S^z_i S^z_j>, S^z_i = (n_i,up - n_i,dn)/2 and
 * eps_i = +1 on sublattice A, -1 on B (the paper defers the definition to its
 * supplement).  For PQMC_HONEYCOMB_TV chains E is the energy per site of
 * Eq. (4), docc holds the interaction energy per site
 * V sum_<ij> <(n_i - 1/2)(n_j - 1/2)> / N, and s_afm the CDW structure factor
 * (1/N^2) sum_ij eps_i eps_j <(n_i - 1/2)(n_j - 1/2)>. */
typedef struct {
    double E, E_err;
    double docc, docc_err;
    double sign, sign_err;
    double accept;          /* accepted / proposed flips */
    double max_dG;          /* max |G - G_fresh| over all stabilisations so far */
    long n_meas;            /* measurements used */
    double s_afm, s_afm_err;
} pqmc_obs;

typedef struct pqmc_ctx pqmc_ctx;

/* Create a context running opts->n_chains identical chains of one model.
 * Builds K, e^{-+dtau K}, the trial orbitals P_sigma (host FP64), draws the
 * initial fields with Philox, uploads everything and computes the left stack
 * and G at tau = -1 on the device. Returns PQMC_EINVAL if N_sigma > N,
 * Ltau is odd, Ltau/2 is not a multiple of n_stab, or the trial shell is open
 * (gap below 1e-8). *out is NULL on failure. */
pqmc_status pqmc_init(const pqmc_lattice* lattice, double U, double dtau, double two_theta,
                      const pqmc_trial* trial, const pqmc_opts* opts, pqmc_ctx** out);

/* Same for a batch of n chains with their own specs (uneven sizes allowed):
 * chain c follows specs[c] and uses Philox chain index chain_offset + c.
 * opts->n_chains is ignored. */
pqmc_status pqmc_init_batch(int n, const pqmc_chain_spec* specs, const pqmc_opts* opts,
                            pqmc_ctx** out);

/* Enqueue n_sweeps sweeps of every chain on the context's stream
 * (asynchronous). measure != 0 records one measurement per sweep and chain.
 * All chains run in one launch; the first call with a given (n_sweeps,
 * measure) captures that launch (and the advance of the device-side sweep
 * index) in a CUDA graph, later calls replay it. */
pqmc_status pqmc_sweep(pqmc_ctx* ctx, int n_sweeps, int measure);

/* Wait for the context's stream and report any device-side error. */
pqmc_status pqmc_synchronize(pqmc_ctx* ctx);

/* Estimates for one chain (chain >= 0) or pooled over all chains (chain = -1,
 * meaningful when the chains share one spec). Synchronises first. */
pqmc_status pqmc_measure(pqmc_ctx* ctx, int chain, pqmc_obs* out);

/* Raw per-sweep records of one chain: out[m*6 + {0..5}] = (sign of the weight
 * from the stabilised stacks, E/site, docc/site, kinetic energy/site, running
 * product of sgn(R) over accepted flips, S_AFM of this configuration) for
 * m < *n; on entry *n is the capacity in records, on return the number
 * written. Synchronises first. */
pqmc_status pqmc_get_measurements(pqmc_ctx* ctx, int chain, double* out, long* n);

/* Latest measurement record of every chain in one device-to-host copy:
 * out[c*6 + {0..5}] as in pqmc_get_measurements (n_chains x 6 doubles; NaN
 * for a chain that has no record yet). Synchronises first. */
pqmc_status pqmc_get_last_records(pqmc_ctx* ctx, double* out);

/* Replace the fields of one chain ((Ltau+2) x fields-per-slice int8, values +-1) and rebuild its
 * stacks and G as at initialisation. Allowed only when an even number of
 * sweeps has been run (the next sweep goes up). */
pqmc_status pqmc_set_fields(pqmc_ctx* ctx, int chain, const int8_t* fields);
pqmc_status pqmc_get_fields(pqmc_ctx* ctx, int chain, int8_t* fields);

/* Current G of one chain and spin as FP64 N x N (after an even number of
 * sweeps: G(tau = -1); after an odd number: G(tau = Ltau+1)). */
pqmc_status pqmc_get_green(pqmc_ctx* ctx, int chain, int spin, double* out);

/* G_sigma at the stabilisation point tau = b * n_stab (b = 0 .. Ltau/n_stab),
 * recomputed from the chain's current fields by the context's own kernels:
 * the right stack B_tau ... B_0 P and the left stack P^T B_{Ltau+1} ...
 * B_{tau+1}, each QR-factorised every n_stab slices, then
 * G = 1 - B_R (B_L B_R)^{-1} B_L as at a stabilisation (the equal-time Green's
 * function of the Method section, both Gutzwiller slices included). The
 * chain's state (stacks, G, counters) is kept aside in a temporary device
 * buffer and put back, so the Markov chain is not disturbed. out: FP64 N x N row-major. Synchronises.
 * PQMC_EINVAL for b out of range; PQMC_ENOMEM if the temporary buffer cannot
 * be allocated. */
pqmc_status pqmc_get_green_at(pqmc_ctx* ctx, int chain, int spin, int b, double* out);

/* Checkpoint of every chain's Markov-chain state: fields, G, both stacks and
 * their log-determinants, counters and running sign, measurement records,
 * stabilisation-error history, accept log, and the sweep index. With
 * buf == NULL, *len receives the size in bytes and nothing is copied;
 * otherwise *len is the capacity of buf (PQMC_EINVAL, with *len set to the
 * size, when it is too small) and on return the bytes written. The caller
 * owns buf. Synchronises; returns the context's sticky error, if any,
 * instead of writing. The format is this library's own (a versioned header,
 * then raw little-endian device contents). */
pqmc_status pqmc_checkpoint(pqmc_ctx* ctx, void* buf, size_t* len);

/* Load a checkpoint into a context created with the same chain specs and the
 * same precision, n_stab, delay_k, seed, chain_offset, max_meas and
 * accept_log (cta_threads and dense_chains may differ: they do not change the
 * results). Later sweeps then continue the checkpointed run exactly: the same
 * Philox draws, accept decisions, G and records. Clears a sticky
 * PQMC_ESTAB / PQMC_ENAN / PQMC_ETIMEOUT of the context, so a failed run
 * can resume from its last good checkpoint. PQMC_EINVAL (nothing loaded) when
 * the data is not a checkpoint of this library or was taken from a context
 * that differs in any of the above. Synchronises. */
pqmc_status pqmc_restore(pqmc_ctx* ctx, const void* buf, size_t len);

/* log|det(B_L B_R)| and sign per spin at the last stabilisation of a chain:
 * out[0..3] = (logabs_up, sign_up, logabs_dn, sign_dn). */
pqmc_status pqmc_get_weight(pqmc_ctx* ctx, int chain, double* out);

/* Run log (no counterpart in the paper: bookkeeping of a run).  Appends one
 * JSON line per chain to the text file at `path`: chain and Philox chain
 * index, sites, slices, precision, sweeps done, records, the sign-reweighted
 * means of the chain's records (E/site, docc, S_AFM), the mean weight sign,
 * the acceptance, max |G - G_fresh| and the latest stabilisation's value,
 * stabilisations done, log|det| and sign of each spin's weight at the last
 * stabilisation, the running sign, and the chain's error bits.  Synchronises
 * the context's stream; PQMC_EINVAL when the file cannot be written. */
pqmc_status pqmc_write_run_log(pqmc_ctx* ctx, const char* path);

/* Accept bits (0/1) of the first n proposals of a chain in visiting order
 * (requires opts.accept_log >= n). */
pqmc_status pqmc_get_accept_log(pqmc_ctx* ctx, int chain, uint8_t* out, long n);

/* max |G - G_fresh| at each stabilisation, oldest first, up to *n values
 * (in: capacity, out: written): the propagated G just before the
 * stabilisation against the G rebuilt from the stacks (in the path
 * precision, or in FP64 when opts.dg_fp64 is set). The history keeps the
 * last 4096 values. */
pqmc_status pqmc_get_stab_errors(pqmc_ctx* ctx, int chain, double* out, long* n);

/* SM clock cycles one chain's CTA has spent, as seen by its thread 0, in
 * each phase of its sweeps so far: out[0..15] = (flip decisions,
 * delayed-update products G -= U V, slice wrapping, stack slice products, QR
 * factorisation, rest of the G refresh, measurement, total, forming Q,
 * Q_L^T Q_R, its inverse, G assembly; inside the inverse: pivot steps,
 * eliminations, column restore and log-determinant; and the update vectors
 * U, V of the accepted flips). */
pqmc_status pqmc_get_phase_cycles(pqmc_ctx* ctx, int chain, long long* out);

/* Sizes of one chain: out[0..6] = (N, N_up, N_dn, Ltau, n_stab, delay_k,
 * fields per slice: N, or 3N/2 bonds for PQMC_HONEYCOMB_TV). */
pqmc_status pqmc_get_dims(pqmc_ctx* ctx, int chain, int* out);

/* Number of chains in the context, or -1 for NULL. */
int pqmc_num_chains(const pqmc_ctx* ctx);

/* Bytes of device memory held by the context, or 0 for NULL. */
size_t pqmc_device_bytes(const pqmc_ctx* ctx);

/* Bytes copied from host memory into the context's device memory at
 * creation (model tables, trial orbitals, initial fields, chain states; the
 * rest of the arena is cleared on the device), or 0 for NULL. */
size_t pqmc_upload_bytes(const pqmc_ctx* ctx);

/* Device kernels launched by this context so far (all entry points; a sweep
 * graph replay counts its two kernels). */
long pqmc_launch_count(const pqmc_ctx* ctx);

/* Last error message of a context (or of the last failed pqmc_init* call when
 * ctx is NULL). Never NULL. */
const char* pqmc_last_error(const pqmc_ctx* ctx);

/* Release the context and its device memory. NULL is allowed. */
void pqmc_free(pqmc_ctx* ctx);

/* Host-side model set-up, exposed for tests (no GPU needed). Builds the
 * hopping matrix K (N x N, row-major) of a lattice, e^{sign_x * dtau K}
 * (dtau < 0 gives e^{+|dtau| K}) and the trial orbitals of one spin
 * (spin 0 up, 1 down; N x n_sigma, row-major) from the library's own FP64
 * symmetric eigensolver. Any output pointer may be NULL. gap receives the
 * gap above the last occupied trial level. */
pqmc_status pqmc_host_model(const pqmc_lattice* lattice, double dtau, const pqmc_trial* trial,
                            int spin, double* K, double* expK, double* P, double* gap);

/* Library's own FP64 symmetric eigensolver (Householder tridiagonalisation +
 * implicit QL with Wilkinson shifts): A is n x n row-major symmetric;
 * eigenvalues ascending into w, eigenvectors as columns of V (row-major).
 * Exposed for tests. */
pqmc_status pqmc_host_eigh(int n, const double* A, double* w, double* V);

/* Result of pqmc_autotune: the pick and every candidate's time. */
typedef struct {
    int delay_k;            /* picked delayed-update block (sites) */
    int cta_threads;        /* picked threads per chain CTA */
    double ms_per_sweep;    /* the pick's time per sweep of the proxy batch */
    int proxy_ltau;         /* interaction slices per chain of the proxy batch */
    int n_candidates;
    int cand_delay_k[32];
    int cand_cta_threads[32];
    double cand_ms[32];     /* ms per sweep of each candidate on the proxy batch (NaN: did not run) */
    int from_cache;         /* 1: the pick came from the cache, no timing was run */
} pqmc_tune;

/* Autotuner of the launch shape (no counterpart in the paper: it picks how
 * the GPU runs the sweep, not what the sweep computes).  For the batch
 * (n, specs) with opts' precision and n_stab it times every candidate
 * delayed-update block (8, 16, 32, 64 sites; only opts->delay_k when that is
 * nonzero) and CTA shape (64/128/256 threads for FP64, 64/128/256/512 for the
 * reduced paths; only opts->cta_threads when nonzero; 64/128 with
 * dense_chains) and returns the fastest.  The timing runs on a proxy batch:
 * the same chains with the projection shortened to proxy_ltau interaction
 * slices (the smallest multiple of 2 n_stab that is >= 8, or the chain's own
 * Ltau when shorter), one warm-up and two timed sweeps per candidate (CUDA
 * events on the context's stream).  The pick is cached per process under a
 * key made of the precision, n_stab, the fixed options and the multiset of
 * chain shapes (N, N_up, N_dn, Ltau, model); with the environment variable
 * PQMC_AUTOTUNE_CACHE naming a file, the cache is also read from and written
 * to that file as JSON.  pqmc_init / pqmc_init_batch call this when
 * opts->delay_k is 0.  Allocates a temporary context (device memory).
 * PQMC_EINVAL for bad specs or options, PQMC_ECUDA when no candidate ran. */
pqmc_status pqmc_autotune(int n, const pqmc_chain_spec* specs, const pqmc_opts* opts, pqmc_tune* out);

/* Launch shape of a context: out[0..3] = (delayed-update block in sites,
 * threads per chain CTA, chain CTAs per SM the kernel is built for, shared
 * memory bytes offered to a chain that keeps G and its scratch resident; a
 * chain whose footprint is larger keeps them in global memory). */
pqmc_status pqmc_get_launch(pqmc_ctx* ctx, int* out);

/* Micro-benchmarks of the arithmetic pipes that bound the sweep (no
 * counterpart in the paper: they measure the GPU the library runs on).  On
 * the current device: out[0] FP64 FMA TFLOP/s over all SMs, out[1] FP64
 * tensor-core (mma.sync m8n8k4 f64) TFLOP/s, out[2] FP32 FMA TFLOP/s,
 * out[3..5] clock cycles of one dependent FP64 FMA, add + divide, and
 * add + square root, out[6..9] clock cycles per FP64 warp instruction of one
 * warp with 1, 8, 16 and 32 active lanes (8 independent chains per lane),
 * out[10] SM count, out[11] the reported SM clock in MHz, out[12] FP64
 * TFLOP/s of a launch whose warps alternate between the FMA and the
 * tensor-core loop, out[13] its time over the mean of the two pure launches
 * (1: the two share one pipe; 0.5: they run side by side); out must hold 14
 * doubles.  Allocates and
 * frees a small device buffer; synchronises the device.  PQMC_ECUDA on a
 * CUDA failure. */
pqmc_status pqmc_probe_pipes(double* out);

/* Test hook of the tensor-core split-BF16 product the BF16X3 path uses for
 * chains kept in global memory (no counterpart in the paper): one CTA
 * computes C = A B with A and B split into BF16 hi + lo parts and the three
 * products A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 by tcgen05
 * MMAs in tensor memory.  Device pointers: A is M x K row-major (trans_a = 0)
 * or K x M row-major holding A^T (trans_a != 0), B is K x N row-major, C is
 * M x N row-major (written).  1 <= M, N, K <= 4096.  Runs on `stream`
 * (NULL: the legacy default stream) and synchronises it.  PQMC_ETIMEOUT when
 * the bounded wait for the tensor cores' completion gave up. */
pqmc_status pqmc_test_tc_gemm(int M, int N, int K, const float* d_A, int trans_a, const float* d_B, float* d_C,
                              void* stream);

/* Error bar of the sign-reweighted estimator <s O>/<s> of the Method
 * section, as pqmc_measure computes it: the records are split into n_groups
 * groups (bins of consecutive sweeps of one chain, or whole chains when
 * pooling), group g contributing the sums sO[g] = sum s O and s[g] = sum s.
 * mean = sum_g sO[g] / sum_g s[g]; the delete-one-group jackknife takes
 * r_g = (sum sO - sO[g]) / (sum s - s[g]) and
 * err = sqrt((n_groups - 1) / n_groups * sum_g (r_g - mean_g r)^2), NaN for
 * n_groups < 2.  Host arrays of n_groups doubles; no GPU needed (exposed for
 * tests).  PQMC_EINVAL for n_groups < 1 or a NULL pointer. */
pqmc_status pqmc_host_jackknife(int n_groups, const double* sO, const double* s, double* mean, double* err);

/* Test hook for the failure path: marks chain `chain` as failed with
 * `code` (PQMC_ENAN or PQMC_ESTAB) exactly as a sweep kernel that met a NaN
 * or a singular pivot would, by writing the kernels' error bits into the
 * chain's device counters and into the context's device error word from the
 * host.  No kernel runs and no GPU fault is involved.  The next
 * pqmc_synchronize / pqmc_sweep / pqmc_checkpoint returns `code` and the
 * context stays failed until pqmc_restore.  Synchronises.  PQMC_EINVAL for a
 * bad chain index or code. */
pqmc_status pqmc_inject_error(pqmc_ctx* ctx, int chain, int code);

/* Allocation-free initialisation of one chain.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory, for example code that runs inside a host
 * application whose device memory is reserved up front by its own allocator,
 * or a loop that must not call cudaMalloc because of the implicit device
 * synchronisation and the failure mode it brings.  It computes, for the FP64
 * path, what pqmc_init_batch + pqmc_set_fields + pqmc_get_green /
 * pqmc_get_weight compute for one chain: the left stack and G at tau = -1
 * for the given fields, with the same kernel.
 *
 *   spec     host pointer, one chain of a Hubbard lattice (validated as in
 *            pqmc_init_batch; PQMC_HONEYCOMB_TV is rejected)
 *   n_stab   slices between QR stabilisations (Ltau/2 must be a multiple)
 *   d_fields device pointer, (Ltau+2) x N int8 fields in {-1,+1}, read only
 *   d_G      device pointer, output, 2 x N x N FP64: G_up then G_dn, row-major
 *   d_logw   device pointer, output, 4 FP64: (logabs_up, sign_up, logabs_dn, sign_dn)
 *   stream   cudaStream_t to run on (NULL: the legacy default stream)
 *
 * It allocates no device memory: every other buffer the kernel uses lives in
 * one 16 MiB array in the library's device image, which every GPU that loads
 * the library holds until the process exits.  A chain needing more than
 * 16 MiB (roughly N > 128 at Ltau = 200, n_stab = 10) is rejected with
 * PQMC_EINVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  All calls share the array and it keeps the last
 * call's contents (each call re-initialises what it reads), so calls that
 * overlap on the GPU, from any stream or thread, race: serialise them.  The
 * call synchronises `stream` before it returns and reports PQMC_ESTAB /
 * PQMC_ENAN / PQMC_ECUDA like the other entry points (message:
 * pqmc_last_error(NULL)). */
pqmc_status pqmc_green_noalloc(const pqmc_chain_spec* spec, int n_stab, const int8_t* d_fields,
                               double* d_G, double* d_logw, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PQMC_H */
