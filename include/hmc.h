/*
 * hmc.h -- C ABI of the GB300 (sm_103a) library for the hot path of Hybrid
 * Monte Carlo on the honeycomb Hubbard model (arXiv:2210.06874, §2).
 *
 * The operator.  Lattice: L x L unit cells of the honeycomb lattice, two
 * sites each, V = 2 L^2 sites, periodic (§1, Fig. 1; §4).  With delta =
 * beta / Nt, h the nearest-neighbour adjacency and E = exp(delta*kappa*h)
 * (E = exp(delta*(kappa*h - mu)) at a chemical potential mu, see
 * hmc_params), the fermion matrix on space-time vectors psi[t][x] is
 *
 *     (M psi)_t     = psi_t - s_t     * E diag(exp(i phi_{t-1})) psi_{t-1}
 *     (M^dag psi)_t = psi_t - s_{t+1} * diag(exp(-i phi_t)) E psi_{t+1}
 *     s_0 = -1 (antiperiodic time boundary), s_t = +1 otherwise, t mod Nt
 *
 * i.e. the transfer-matrix (exponential-hopping) form of the fermion
 * operator whose linear form is printed as Eq. (2.2).  phi is the phase
 * angle: phi = delta * phi_paper, so the bosonic action of Eq. (2.1) reads
 * sum(phi^2) / (2 delta U).
 *
 * Layouts (all arrays time-major, site index fastest):
 *   phi, pi, F   double  [Nt][V]
 *   complex128   double2 [Nt][V]   interleaved (re, im)  == torch.complex128
 *   complex64    float2  [Nt][V]   interleaved (re, im)  == torch.complex64
 *   site x = s*L*L + m1*L + m2 (s = 0: sublattice A, s = 1: sublattice B);
 *   the A site of cell (m1,m2) bonds to the B sites of cells (m1,m2),
 *   (m1-1,m2), (m1,m2-1), indices mod L.
 *
 * Ownership.  Every array pointer is caller-owned DEVICE memory (e.g. a
 * torch tensor's data_ptr()) unless named *_host; the library never frees
 * or retains it past the call.  hmc_ctx owns only derived data: E in FP64
 * and its FP16 split, solver workspaces and the device status words.
 * `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 * return results in host structs (stats, out) synchronise that stream;
 * the others are asynchronous.  One context serves one stream at a time:
 * its workspaces are shared by all calls on it.
 *
 * Errors.  Every entry point returns an hmc_status.  Argument checks happen
 * on the host before any launch.  Device-side failures (non-finite
 * reductions, solver not converged, a bounded wait that gave up) are
 * recorded in a device status word and reported by the next synchronising
 * call on the context.  No call traps or aborts the GPU context.
 */
#ifndef HMC_GB300_H
#define HMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hmc_status {
    HMC_OK = 0,
    HMC_ERR_BAD_ARG = -1,           /* invalid size, pointer or parameter */
    HMC_ERR_CUDA = -2,              /* a CUDA runtime call failed */
    HMC_ERR_CG_NOT_CONVERGED = -3,  /* max_iter reached above tolerance */
    HMC_ERR_NONFINITE = -4,         /* NaN/Inf seen in a reduction */
    HMC_ERR_TIMEOUT = -5,           /* a bounded device wait gave up */
    HMC_ERR_UNSUPPORTED = -6        /* sizes beyond what a kernel supports */
} hmc_status;

typedef enum hmc_precision {
    HMC_PREC_FP64 = 0,   /* every step in FP64 on CUDA cores */
    HMC_PREC_MIXED = 1   /* FP16-split tensor-core contraction, FP32 CG with
                            FP64 reliable updates; FP64 for residuals, sums,
                            force and Metropolis */
} hmc_precision;

/* Physics and solver parameters of one Markov chain. */
typedef struct hmc_params {
    int L;               /* unit cells per direction, 1 <= L; V = 2 L^2 */
    int Nt;              /* time slices, >= 1 */
    double kappa;        /* hopping amplitude of Eq. (1.1) */
    double U;            /* on-site coupling of Eq. (1.1), > 0 */
    double beta;         /* inverse temperature; delta = beta / Nt */
    int n_md;            /* leapfrog steps per trajectory, >= 1 */
    double traj_length;  /* trajectory length tau; eps = tau / n_md */
    double cg_tol;       /* target |chi - M M^dag x| / |chi| (FP64 true residual) */
    int cg_max_iter;     /* CG iteration cap per solve */
    int precision;       /* hmc_precision used by hmc_trajectory */
    double ru_delta;     /* mixed CG: reliable update when |r| < ru_delta * max|r|
                            since the last update (0 selects the default,
                            0.05) */
    int team_ctas;       /* CTAs of a persistent launch (0: automatic); in a
                            batch, 2..8 runs the chain on a thread-block
                            cluster of that many CTAs (one size per batch;
                            those chains go first), else one CTA */
    int tile_slices;     /* time slices per tensor-core tile, one of 8, 16, 32
                            (operand_mode 4: 1..64; 0: automatic) */
    int inner_ctas;      /* CTAs running the FP32 iterations of the mixed CG
                            (0: automatic; the FP64 steps use all CTAs) */
    int operand_mode;    /* mixed path: 0 automatic, 1 stream E through shared
                            memory on every application, 2 keep each CTA's rows
                            of E resident for the whole solve (needs
                            V <= 256 and one CTA per 128-site block; a chain
                            with V <= 128 then keeps its FP32 CG vectors in
                            shared memory too when they fit), 3 run the FP32
                            iterations on the CUDA cores of one thread-block
                            cluster of inner_ctas CTAs (1..16; 0 picks the
                            largest of 16, 8, 4, 2, 1 that fits), with E^T
                            in FP32 and the iterates of each CTA's time
                            slices in its shared memory: needs at most 16
                            slices per CTA and the layout within the shared
                            memory of a CTA (about V <= 128 at 8 slices);
                            HMC_ERR_UNSUPPORTED otherwise, or if the device
                            refuses the cluster (sizes above 8 are
                            non-portable), 4 slice-major tensor-core tiles:
                            up to 64 time slices (x re/im) as the MMA's
                            M = 128 and up to 288 sites as its N, E
                            streamed, one FP32 accumulator of a scaled
                            FP16 split (any V) */
    int cluster_mode;    /* mixed path, inner team of 2..8 CTAs: 0 automatic
                            (launch it as one thread-block cluster, whose
                            barriers and sums go through distributed shared
                            memory, when the launch accepts the cluster; else
                            global-memory barriers), 1 require the cluster
                            (HMC_ERR_UNSUPPORTED if the launch refuses it),
                            2 never.  Resident E accepts inner_ctas as a
                            multiple of the 128-site blocks: the extra CTAs
                            take further slice tiles of the same block. */
    int integrator;      /* molecular dynamics of hmc_trajectory: 0 leapfrog
                            (n_md steps, n_md + 1 force evaluations), 1 the
                            second-order minimum-norm integrator of Omelyan,
                            Mryglod and Folk (2003), lambda = 0.19318...
                            (n_md steps, 2 n_md + 1 force evaluations, a
                            much smaller energy violation at equal step) */
    double mu;           /* chemical potential (the sign-problem setting of
                            the paper's section on tensor networks, where
                            p ~ det(M[phi,mu] M[phi,-mu]^dag)), the mu of
                            the particle-hole Hamiltonian's term
                            + mu sum_x rho_x: M[phi,mu] is the particles'
                            matrix, E = exp(delta (kappa h - mu)) =
                            e^{-delta mu} exp(delta kappa h), in every
                            operator of the context (not in the Eq. (2.2)
                            operator of hmc_apply_brs); 0 = half filling */
    int ru_every;        /* mixed CG: a reliable update at the latest after
                            this many FP32 iterations (0 selects 1000), so a
                            stalled FP32 recursion still reaches an FP64
                            residual check; two checks in a row that do not
                            halve the true residual switch the rest of the
                            solve to FP64 CG iterations */
    double hb_gamma;     /* mass preconditioning (Hasenbusch, Phys. Lett. B 519
                            (2001) 177): hop factor g in [0, 1) of the heavy
                            operator M_g = 1 - g S E D (used when hb_inner > 0) */
    int hb_inner;        /* 0: one pseudofermion (the plain HMC of §2); 1..64:
                            hmc_trajectory uses two pseudofermions, chi_1 for
                            det(M_g M_g^dag) and chi_2 for det(M M^dag) /
                            det(M_g M_g^dag), on a two-level leapfrog (Sexton
                            and Weingarten, Nucl. Phys. B 380 (1992) 665): n_md
                            outer steps for the ratio force, hb_inner inner
                            steps per outer step for the bosonic and heavy
                            forces.  The same target density.  FP64, or mixed
                            precision with operand_mode 5 (split-K tiles, whose
                            epilogues scale the contraction by g; other mixed
                            operand modes return HMC_ERR_UNSUPPORTED); FP64
                            solves start from zero, mixed ones after the first
                            of each level from that level's previous
                            solution; integrator must be 0 */
} hmc_params;

typedef struct hmc_cg_stats {
    int iterations;          /* CG iterations (inner iterations for MIXED) */
    int reliable_updates;    /* FP64 residual recomputations (MIXED) */
    double true_residual;    /* |chi - M M^dag x| / |chi| in FP64 */
    int status;              /* hmc_status of the solve */
    int fp64_iterations;     /* MIXED: FP64 CG iterations after a stall (0 normally) */
} hmc_cg_stats;

typedef struct hmc_traj_out {
    double dH;               /* H(end) - H(start), Eq. (2.1) */
    double H0, H1;
    double u;                /* Metropolis uniform drawn for this trajectory */
    int accept;              /* 1 if u < exp(-dH) */
    int cg_iterations;       /* summed over the n_md + 1 solves */
    int cg_solves;
    int reliable_updates;
    double max_true_residual;
    int status;
    int fp64_iterations;     /* MIXED: FP64 CG iterations of stalled solves */
    int cg_iterations_outer; /* mass preconditioning: the ratio solves' share of
                                cg_iterations (0 otherwise) */
    int cg_solves_outer;     /* ... and of cg_solves */
} hmc_traj_out;

typedef struct hmc_ctx hmc_ctx;

/* Build h and E = exp(delta*(kappa*h - mu)) (FP64, plus its FP16 hi/lo split for
 * the MIXED path) for the lattice in *p and allocate workspaces on the
 * current CUDA device.  *out receives the context.
 * Errors: HMC_ERR_BAD_ARG (L < 1, Nt < 1, U <= 0, ...), HMC_ERR_CUDA. */
int hmc_ctx_create(const hmc_params* p, hmc_ctx** out);

/* Free everything the context owns.  NULL is accepted. */
int hmc_ctx_destroy(hmc_ctx* ctx);

/* Copy the FP64 transfer matrix E (V x V, row-major) to host memory. */
int hmc_get_transfer_matrix(hmc_ctx* ctx, double* E_host, size_t n_elems);

/* psi_out = M[phi] psi_in  (definition above; Eq. (2.2) in exponential
 * form).  prec = HMC_PREC_FP64: psi_in/psi_out complex128; FP64 CUDA-core
 * contraction.  prec = HMC_PREC_MIXED: psi_in/psi_out complex64; FP16-split
 * tensor-core contraction with FP32 accumulation.  psi_out must not alias
 * psi_in.  Asynchronous on `stream`. */
int hmc_apply_M(hmc_ctx* ctx, const double* phi, const void* psi_in, void* psi_out,
                int prec, void* stream);

/* psi_out = M^dag[phi] psi_in; layouts and precision as hmc_apply_M. */
int hmc_apply_Mdag(hmc_ctx* ctx, const double* phi, const void* psi_in, void* psi_out,
                   int prec, void* stream);

/* Solve (M M^dag) x = chi (Eq. (2.1)'s pseudofermion kernel) by conjugate
 * gradients from x0 = 0.  chi and x are complex128 [Nt][V].  prec FP64:
 * plain CG, stop on the recursive residual.  prec MIXED: FP32 CG on the
 * tensor-core operator with FP64 reliable updates; stops on the FP64 true
 * residual.  Both report the final FP64 true residual in *stats (host
 * struct; the call synchronises `stream`).  Returns
 * HMC_ERR_CG_NOT_CONVERGED if max_iter was hit (x holds the last iterate). */
int hmc_cg_solve(hmc_ctx* ctx, const double* phi, const void* chi, void* x,
                 double tol, int max_iter, int prec, hmc_cg_stats* stats, void* stream);

/* F = dS/dphi for S = sum(phi^2)/(2 delta U) + chi^dag (M M^dag)^{-1} chi,
 * given the kept solve x = (M M^dag)^{-1} chi (complex128):
 *     F = phi / (delta U) + 2 Im(x * conj(M^dag x))    (FP64).
 * Asynchronous. */
int hmc_force(hmc_ctx* ctx, const double* phi, const void* x, double* F, void* stream);

/* S = sum(phi^2) / (2 delta U) + Re(chi^dag x): the action of Eq. (2.1)
 * without the momenta, given x = (M M^dag)^{-1} chi from hmc_cg_solve (so
 * the second term is chi^dag (M M^dag)^{-1} chi).  Deterministic FP64
 * reduction; *S_host is a host pointer and the call synchronises `stream`.
 * Returns HMC_ERR_NONFINITE if S is not finite. */
int hmc_action(hmc_ctx* ctx, const double* phi, const void* chi, const void* x, double* S_host,
               void* stream);

/* One HMC trajectory (§2) on device field phi (in/out, double [Nt][V]):
 * momenta pi ~ exp(-pi^2/2) and noise rho ~ exp(-rho^dag rho) from Philox
 * streams (seed, traj_index, chain), chi = M rho, n_md molecular-dynamics
 * steps of params.integrator (leapfrog or the minimum-norm integrator; drift
 * phi += c*eps*delta*pi, kick pi -= c*eps*delta*dS/dphi), Metropolis
 * with u from the generator.  On rejection phi is restored.  The whole
 * trajectory runs in one persistent launch; *out (host) is filled and the
 * stream synchronised.  Precision: params.precision. */
int hmc_trajectory(hmc_ctx* ctx, double* phi, uint64_t seed, uint64_t traj_index,
                   uint32_t chain, hmc_traj_out* out, void* stream);

/* ---- Observables (M^{-1} sources) ---------------------------------------
 * Zero-momentum single-particle correlator on sublattice A, the correlator
 * whose decay in Euclidean time gives the single-particle gap (§2): source
 * b = V_A^{-1/2} on the A sites (x < V/2) of slice 0; g = M^{-1} b =
 * M^dag (M M^dag)^{-1} b (CG to tol in `precision`, then the FP64 M^dag);
 * C[t] = V_A^{-1/2} sum_{x < V/2} g_t(x), t = 0..Nt-1.  phi: device double
 * [Nt][V]; C: device complex double [Nt]; stats as for hmc_cg_solve (and
 * its status codes).  Allocates 3 V Nt complex doubles on `stream` for the
 * call (stream-ordered).  The gap fit itself is analysis, not done here. */
int hmc_correlator_k0(hmc_ctx* ctx, const double* phi, double tol, int max_iter, int precision,
                      void* C, hmc_cg_stats* stats, void* stream);

/* Staggered spin traces of G = M[phi]^{-1} by Z2 noise, the ingredients of
 * the staggered magnetisation that §2 names as an order parameter (its
 * estimator is cited there, not printed).  With eps_x = +1 on sublattice A
 * (x < V/2), -1 on B, on every slice:
 *     T_s = tr(eps G),  T_u = tr(G),  T_ss = tr(eps G eps G).
 * Sample k uses eta_k(e) = 1 - 2 (word0 & 1), word0 the first Philox word of
 * element e = t V + x, stream 4, counter (e, 4, k, chain), key `seed`;
 * v = M^{-1} eta_k and w = M^{-1} (eps v), each M^{-1} = M^dag (M M^dag)^{-1}
 * (CG to tol in `precision`, then the FP64 M^dag); the sample's estimates
 * are (eta^T eps v, eta^T v, eta^T eps w), unbiased for the three traces.
 * In the particle-hole basis of §1 (spin up = particles, spin down = holes,
 * whose propagator is conj(G) at mu = 0), Wick's theorem gives the staggered
 * space-time susceptibility of the field, chi_s = (Re T_u - Re T_ss) / (2N),
 * N = V Nt, which this call also returns.
 *   n_noise  1 .. 2^20 samples
 *   samples  device complex128 [n_noise][3] (T_s, T_u, T_ss per sample), or NULL
 *   mean     device complex128 [4]: the sample means of T_s, T_u, T_ss, and
 *            (chi_s of the means, 0)
 *   stats    host: iterations, reliable updates and FP64 iterations summed
 *            over the 2 n_noise solves, the largest true residual, the status
 * Sums are FP64 in a fixed order (repeatable bit for bit).  A context with
 * mu != 0 returns HMC_ERR_UNSUPPORTED (the holes' propagator is conj(G) only
 * at mu = 0); solver failures return their status (e.g.
 * HMC_ERR_CG_NOT_CONVERGED) and stop.  Allocates 5 V Nt + 3 n_noise complex
 * doubles and 1536 doubles on `stream` for the call (stream-ordered) and
 * synchronises `stream` before returning. */
int hmc_spin_traces(hmc_ctx* ctx, const double* phi, int n_noise, uint64_t seed, uint32_t chain,
                    double tol, int max_iter, int precision, void* samples, void* mean,
                    hmc_cg_stats* stats, void* stream);

/* ---- The printed operator, Eq. (2.2) -------------------------------------
 * The mixed-differencing (Brower-Rebbi-Schaich) fermion operator exactly as
 * Eq. (2.2) prints it, as a sparse stencil; no context needed.  With
 * dk = delta*kappa and phi the phase angle (delta * phi_paper):
 *   A site: (M psi)_{x,t} = psi_{x,t+1} - e^{+i phi_{x,t}} psi_{x,t} - dk sum_<y> psi_{y,t}
 *   B site: (M psi)_{x,t} = psi_{x,t} - e^{-i phi_{x,t}} psi_{x,t-1} - dk sum_<y> psi_{y,t}
 * antiperiodic in time; dagger = 1 applies the adjoint.  Layouts as above
 * (time-major [Nt][V], site x = s*L*L + m1*L + m2). */

/* Phase tables for hmc_apply_brs: cis64 (complex128, may be NULL) and cis32
 * (complex64, may be NULL) = exp(i phi), device arrays of 2 L^2 Nt entries.
 * Recompute whenever phi changes.  Asynchronous. */
int hmc_brs_phases(int L, int Nt, const double* phi, void* cis64, void* cis32, void* stream);

/* out = M in (dagger = 0) or M^dag in (dagger = 1) of Eq. (2.2).
 * prec HMC_PREC_FP64: cis, in, out complex128; HMC_PREC_MIXED: complex64
 * (FP32 arithmetic).  out must not alias in.  2 L^2 Nt < 2^31, Nt <= 65535.
 * Asynchronous. */
int hmc_apply_brs(int L, int Nt, double delta_kappa, const void* cis, const void* in, void* out,
                  int prec, int dagger, void* stream);

/* ---- Batched chains ----------------------------------------------------
 * Many independent Markov chains, each with its own hmc_params (lattice
 * size, Nt, U, beta, ...), advanced together: one persistent launch where
 * every CTA takes the next chain from a work queue (largest first) and runs
 * its whole trajectory with the MIXED path (HMC_PREC_MIXED required; other
 * precisions return HMC_ERR_UNSUPPORTED).  Chains with equal L and
 * delta*kappa share E.  The launch is captured once into a CUDA graph on
 * the batch's own stream and replayed; it is ordered after `stream`.
 * Chain i uses Philox chain id i. */
typedef struct hmc_batch hmc_batch;

/* params: host array of n_chains parameter sets (mixed precision).  Chains
 * with team_ctas >= 2 run as thread-block-cluster teams of that many CTAs
 * (all such chains of a batch must ask for the same size, at most 8;
 * HMC_ERR_UNSUPPORTED otherwise, or if the chain's launch shape cannot use
 * all of them as one inner team). */
int hmc_batch_create(const hmc_params* params, int n_chains, hmc_batch** out);
int hmc_batch_destroy(hmc_batch* batch);

/* Packed field layout: chain i occupies phi[offsets[i] .. offsets[i+1]) as
 * double [Nt_i][V_i]; offsets (host, n_offsets >= n_chains + 1) is filled. */
int hmc_batch_layout(const hmc_batch* batch, int64_t* offsets, int n_offsets);

/* One trajectory of every chain on the packed device field phi (in/out).
 * out: host array of n_chains records; the call synchronises.  Returns the
 * first non-OK chain status (each record carries its own). */
int hmc_batch_trajectory(hmc_batch* batch, double* phi, uint64_t seed, uint64_t traj_index,
                         hmc_traj_out* out, void* stream);

/* Philox4x32-10 draws of the library's streams, for checking the generator
 * (Salmon et al., SC'11): element e of stream `stream_id` for
 * (seed, traj, chain) -> raw[4e..4e+3] (uint32, may be NULL) and the
 * Box-Muller pair z0[e], z1[e] (double, may be NULL).  Device pointers;
 * n >= 0 elements.  Asynchronous. */
int hmc_rng_draw(uint64_t seed, uint32_t stream_id, uint64_t traj, uint32_t chain,
                 int64_t n, uint32_t* raw, double* z0, double* z1, void* stream);

/* FP64 CG solve of (M M^dag) x = chi that allocates no device memory.
 *
 * The paper has no counterpart; this is a library convenience.  Callers that
 * may not call cudaMalloc -- hosts whose device memory comes from a
 * framework pool or a fixed real-time budget, plugins barred from growing
 * the device heap -- cannot create an hmc_ctx.  This call needs none: it
 * runs the same FP64 CG as hmc_cg_solve with HMC_PREC_FP64 (same algorithm,
 * stopping rule and stats), with its scratch in one static device array of
 * about 2.1 MB that every GPU which loads the library holds until the
 * process exits.
 *
 *   E      device, double [V][V], the transfer matrix exp(delta*kappa*h),
 *          row-major and exactly symmetric (e.g. from hmc_get_transfer_matrix)
 *   L, Nt  lattice: V = 2 L^2 sites, Nt slices; V * Nt must not exceed
 *          32768, larger sizes return HMC_ERR_UNSUPPORTED before any launch
 *   phi    device, double [Nt][V]; chi, x device complex128 [Nt][V]
 *   stats  host; the call synchronises `stream`
 *
 * The call copies its statistics to the host and synchronises the stream,
 * so it cannot be recorded into a CUDA graph: on a stream that is being
 * captured it returns HMC_ERR_UNSUPPORTED before enqueuing anything, and the
 * capture stays valid.  The first call on each device (and the first after
 * that device's context was replaced, e.g. by cudaDeviceReset) looks up the
 * array's device address (cudaGetSymbolAddress) with that device current.
 * Every call on a device shares the one array: calls that overlap on the
 * GPU (other streams, other host threads) race and give wrong results;
 * serialise them.  The barrier, status and output words are cleared on
 * every call.  Errors as hmc_cg_solve. */
int hmc_cg_solve_noalloc(const double* E, int L, int Nt, const double* phi, const void* chi,
                         void* x, double tol, int max_iter, hmc_cg_stats* stats, void* stream);

/* ---- Bounded waits ---------------------------------------------------------
 * Every spin of the library's kernels (team barriers, mbarrier waits of the
 * tensor-core pipelines, cluster exchanges) gives up after a time limit and
 * records HMC_ERR_TIMEOUT, which the next synchronising call returns; the
 * kernel then leaves its waits and frees what it holds, so the context stays
 * usable.  The paper has no counterpart (failure handling of this library).
 *
 * hmc_ctx_set_wait_limit: the limit of every wait of kernels launched on
 * this context from now on, in seconds (0 restores the default of 20 s; at
 * most 3600).  A limit shorter than a whole solve makes the CTAs that wait
 * out the FP32 iterations time out: keep the default in normal use.
 * Synchronises the device.
 *
 * hmc_debug_team_padding: host-side fault injection for testing the timeout
 * path.  Every team barrier of this context's later persistent launches
 * expects extra_ctas (0..1024) CTAs more than were launched, so the first
 * one never completes and its bounded wait runs out.  0 restores normal
 * operation. */
int hmc_ctx_set_wait_limit(hmc_ctx* ctx, double seconds);
int hmc_debug_team_padding(hmc_ctx* ctx, int extra_ctas);

/* Library version string (static storage). */
const char* hmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HMC_GB300_H */
