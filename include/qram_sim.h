/*
 * qram_sim.h -- C ABI of the B300 (sm_103a) trajectory simulator for
 * amplitude-damped bucket-brigade QRAM queries with branch pruning.
 *
 * Method: Chen et al., "Classical simulation of amplitude-damped
 * bucket-brigade quantum random access memories via predictable branch
 * evolution" (arXiv 2609.34935).  Every call below names the passage that
 * defines the operation it performs.
 *
 * Conventions shared by all calls
 *   - Tree: nodes v = 0 .. 2^n - 2, layer l(v) = floor(log2(v + 1)),
 *     children 2v+1 (left) and 2v+2 (right); each node has a router slot and
 *     a data slot, site id = 2v + slot (0 = router, 1 = data), M = 2(2^n - 1)
 *     sites (Sec. II.A).  The bit routed at layer l is address bit n-1-l
 *     (most significant bit at the root; leaf ranges of Eq. (7)).
 *   - Schedule: T = 6n + 2k slices; slices 1 .. T-1 carry gates, each
 *     followed by one joint damping layer over all M sites (Sec. II.B).
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed
 *     and counter (c0, c1 | stream << 24, traj_lo, traj_hi).  Stream 1
 *     draws the candidate set of Theorem 3 (sampler version 2): every
 *     (slice, site) pair is a candidate independently with probability
 *     gamma; the pairs, numbered (slice - 1) * M + site, are cut into blocks
 *     of 2048 and the candidates of block g follow from geometric gaps, draw
 *     r being the 64-bit word (0,1) or (2,3) of counter (g, r / 2) and its
 *     gap the greedy 13-bit inverse of 64-bit fixed-point powers of
 *     1 - gamma (q_0 = 2^64 - floor(gamma 2^64), q_{m+1} = q_m^2 / 2^64,
 *     floored).  Stream 2 (c0 = 0, c1 = slice) is the auxiliary draw of each
 *     damping layer, stream 3 (c0 = c1 = 0) the final tree measurement.  A
 *     trajectory is a pure function of (seed, trajectory index, gamma).
 *   - Memory: "host" pointers are read during the call only; "device"
 *     pointers are CUDA global memory owned by the caller.  The library
 *     owns only its scratch, allocated on the device of the simulator.
 *   - Streams: every call is stream-ordered on the stream given at creation
 *     (NULL = legacy default stream).  Calls return once work is enqueued,
 *     except where stated; device-side failures are reported per trajectory
 *     in qram_result_t.status and summarised by qram_sync().
 *   - Errors: every int-returning call returns a QRAM_* code; no call
 *     aborts the process or throws across this boundary.
 */
#ifndef QRAM_SIM_H
#define QRAM_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* candidate sampler implemented by this library (see "Random numbers") */
#define QRAM_SAMPLER_VERSION 2

enum {
    QRAM_OK = 0,
    QRAM_E_ARG = 1,      /* invalid argument (sizes, gamma, duplicate address, norm) */
    QRAM_E_OOM = 2,      /* device or host allocation failed */
    QRAM_E_CUDA = 3,     /* a CUDA runtime call failed */
    QRAM_E_TIMEOUT = 4,  /* a bounded device wait gave up; per trajectory: its cycle budget (2^34) ran out */
    QRAM_E_BUSY = 5,     /* server queue full / resource busy */
    QRAM_E_CAP = 6,      /* a per-trajectory capacity was exceeded (result marked) */
    QRAM_E_STATE = 7,    /* call not valid in the current state */
    QRAM_E_TOOBIG = 8    /* problem exceeds the static scratch of qram_run_static */
};

enum { QRAM_QUTRIT = 0, QRAM_QUBIT = 1 };

/* Noise channel of the layer that follows every slice's gates (see
 * qram_set_channel). */
enum { QRAM_CHANNEL_DAMPING = 0, QRAM_CHANNEL_DEPHASING = 1, QRAM_CHANNEL_HEATING = 2 };

/* One QRAM query problem (Sec. II.A; input class of Sec. IV.D: a coherent
 * superposition over addresses with one bus column per address). */
typedef struct {
    int32_t encoding;          /* QRAM_QUTRIT (Prop. 1) or QRAM_QUBIT (Theorems 1-2) */
    int32_t n, k;              /* 1 <= k <= n <= 14, k <= 8 (the schedule needs k <= n) */
    const uint8_t *memory;     /* host, 2^n cells; bit t of memory[i] is d_i^(t) (Eq. (1)) */
    int32_t num_branches;      /* D, 1 <= D <= 2^n */
    const uint32_t *addr;      /* host, D distinct addresses */
    const uint32_t *bus;       /* host, D bus words < 2^k */
    const double *amp_re;      /* host, D; sum |amp|^2 = 1 within 1e-12 */
    const double *amp_im;      /* host, D */
    uint64_t seed;             /* Philox key */
    uint32_t sampler_version;  /* must be QRAM_SAMPLER_VERSION (geometric-gap candidate draw) */
} qram_problem_t;

/* Per-trajectory result, written by qram_run_pruned / qram_run_full. */
typedef struct {
    double fidelity;            /* |<psi_id,0|psi>|^2/<psi_Q|psi_Q> if the sampled tree
                                   configuration Q is the ground one, else 0 (App. C) */
    double fidelity_unsampled;  /* |<psi_id,0|psi>|^2 / <psi|psi> */
    double p_ground;            /* probability of the ground tree configuration */
    uint32_t bad;               /* B: input branches in the bad union R (Algorithm 1) */
    int32_t ref;                /* reference branch = first good branch, -1 if none */
    uint32_t ncand;             /* candidate sites drawn over all slices */
    uint32_t explicit_comps;    /* components evolved explicitly */
    uint16_t jumps;             /* damping layers whose joint outcome J was non-empty */
    uint16_t first_jump_slice;  /* slice of the first non-empty J, 0 if none */
    uint16_t jump_sites;        /* sum of |J| */
    uint8_t q_ground;           /* 1 if the sampled Q is the ground configuration */
    uint8_t status;             /* QRAM_OK or a QRAM_E_* code for this trajectory */
} qram_result_t;

typedef struct qram_sim qram_sim_t;

/* Create a simulator for one problem on CUDA device `device`, stream
 * `cuda_stream` (a cudaStream_t, may be NULL).  Inputs are validated
 * (QRAM_E_ARG) and copied to the device; the caller keeps ownership of the
 * host arrays.  On success *out owns device memory until qram_sim_destroy. */
int qram_sim_create(const qram_problem_t *problem, int device, void *cuda_stream, qram_sim_t **out);

/* Release everything the simulator owns (waits for its stream). */
void qram_sim_destroy(qram_sim_t *sim);

/* Candidate sampling and classification only (Algorithm 1, steps 1-2;
 * Theorem 3 step 1; Eq. (7) qutrit, Eq. (9) qubit).  For trajectories
 * traj0 .. traj0 + ntraj - 1 with damping rates gamma[t] (device, ntraj):
 *   cand[t * cap + c]  (device, ntraj * cap) packed (slice << 16) | site, in
 *                      increasing (slice, site) order;
 *   ncand[t]           (device) number of candidates (may exceed cap: then
 *                      only cap are written and status is QRAM_E_CAP);
 *   bad_bits[t * W + w] (device, W = ceil(2^n / 32)) bit a of the bitmap is
 *                      set iff address a is in the bad union R;
 *   bad[t], ref[t]     (device) B and the reference branch index (-1: none).
 * Returns QRAM_E_ARG for gamma outside [0, 1) (checked on the device: the
 * affected trajectory gets ncand = 0xFFFFFFFF). */
int qram_sample_faults(qram_sim_t *sim, uint64_t traj0, uint32_t ntraj, const double *gamma,
                       uint32_t cap, uint32_t *cand, uint32_t *ncand, uint32_t *bad_bits,
                       uint32_t *bad, int32_t *ref);

/* Pruned simulation (Algorithm 1): bad branches plus the reference branch
 * are evolved explicitly with the joint damping sampler of Sec. IV.D; the
 * good branches enter the mask weights (Eq. (21)) and the final state
 * through their closed forms (Prop. 1, Eq. (8); Theorem 2, Eq. (16)), and
 * are annihilated once a non-empty jump fires (Sec. VI.A).  gamma: device,
 * ntraj values in [0, gamma_lim); out: device, ntraj results.
 *
 * Damping-rate limit.  Amplitudes are carried unnormalised as a^e with an
 * integer count e of K0 factors (a = sqrt(1 - gamma)); normalisation happens
 * only in ratios.  The weights a^(2e) must stay in the normal FP64 range:
 * gamma_lim = 1 - exp(-650 / ((2n + k)(T - 1))), i.e. 0.255 at n = 12, k = 4
 * and 0.20 at n = 14, k = 4 (the oracle renormalises every layer and has no
 * such limit).  A trajectory whose rate is outside [0, gamma_lim) reports
 * status QRAM_E_ARG; nothing is computed for it.
 *
 * Launch order (no paper counterpart).  With more trajectories than CTAs the
 * run first scores every trajectory's expected cost on the device (its damping
 * candidates of Sec. IV, regenerated from the same fault stream, each weighted
 * by 2^(n - 2L) (T - s) for a candidate at slice s on layer L: the branches a
 * jump there would leave explicit, times its probability, times the slices
 * left), sorts the indices into quarter-octave buckets of descending score
 * (rejected rates last), and the persistent CTAs take them in that order, so
 * that expensive trajectories do not start last.  Scores and permutation live
 * in stream-ordered memory (cudaMallocAsync on the simulator's stream, freed
 * after the launch); if that allocation fails the run keeps index order.
 * Results are the same in either order.  Both runs and graphs
 * (qram_graph_create) do this; qram_launch_count counts the score and sort
 * kernels. */
int qram_run_pruned(qram_sim_t *sim, uint64_t traj0, uint32_t ntraj, const double *gamma,
                    qram_result_t *out);

/* Full simulation: every branch evolved explicitly from the same noise
 * history (the comparison mode of Sec. VI.A).  Same arguments. */
int qram_run_full(qram_sim_t *sim, uint64_t traj0, uint32_t ntraj, const double *gamma,
                  qram_result_t *out);

/* Test hook (fixed noise histories of Sec. VI.A): while set, trajectory
 * traj0 + t of the next runs takes its candidate set from
 * cand[off[t] .. off[t+1]) (device, packed as in qram_sample_faults, sorted)
 * instead of the FAULT stream, for t < nhist; the auxiliary and final draws
 * still come from the Philox streams.  Pass nhist = 0 to clear.  The arrays
 * must stay valid while the hook is set. */
int qram_set_fault_history(qram_sim_t *sim, uint32_t nhist, const uint32_t *cand, const uint32_t *off);

/* Upper bound on the damping rates of the next runs (0 < gmax < gamma_lim of
 * qram_run_pruned, else QRAM_E_ARG), used to
 * size the per-trajectory candidate scratch without reading the rates back
 * to the host; 0 clears it (each run then reduces gamma on the device and
 * synchronises once).  A trajectory whose candidates overflow the sized
 * scratch is reported with status QRAM_E_CAP, never truncated silently. */
int qram_set_gamma_bound(qram_sim_t *sim, double gmax);

/* Limit the persistent launch of this simulator to at most `nctas` CTAs
 * (0 = one slot per resident CTA on every SM, the default).  Scratch memory
 * scales with the number of CTAs; fewer CTAs leave room for other work on
 * the same GPU.  Takes effect at the next run. */
int qram_set_launch_ctas(qram_sim_t *sim, uint32_t nctas);

/* CUDA-graph capture of one persistent batched launch (pruned, mode 0, or
 * full, mode 1) of ntraj trajectories: the graph holds the work-counter reset
 * (with more trajectories than CTAs also the launch-order score and sort,
 * their memory allocated and freed inside the graph) and the trajectory
 * kernel.  The
 * first trajectory index is read from
 * traj0_dev (device, one uint64) when the graph runs, so one graph serves
 * successive batches; gamma (device, ntraj) and out (device, ntraj results)
 * are bound at capture.  Needs a damping-rate bound (qram_set_gamma_bound)
 * so that nothing is read back to the host; the scratch is sized before the
 * capture.  Capture happens on a private stream; qram_graph_launch runs the
 * graph on the simulator's stream.  The graph is valid until the
 * simulator's scratch changes (qram_set_launch_ctas, a larger gamma bound). */
typedef struct qram_graph qram_graph_t;
int qram_graph_create(qram_sim_t *sim, int mode, uint32_t ntraj, const double *gamma, qram_result_t *out,
                      const uint64_t *traj0_dev, qram_graph_t **graph);
int qram_graph_launch(qram_graph_t *graph);
void qram_graph_destroy(qram_graph_t *graph);

/* Mixed persistent launch (batching of concurrent queries; no paper counterpart:
 * the paper runs one query at a time).  One work-stealing launch, captured
 * in a CUDA graph, over the trajectories of several problems of different
 * encodings, address widths n and data widths k: problem q contributes
 * trajectories traj0[q] .. traj0[q] + ntraj[q] - 1 with damping rates
 * gamma[q] (device, ntraj[q]) and results out[q] (device, ntraj[q]); mode 0
 * pruned, 1 full for all.  The global counter runs over the concatenated
 * ranges, so problems with uneven per-trajectory cost share the SMs; each
 * CTA runs Algorithm 1 for one trajectory of one problem at a time, and
 * every trajectory's result is bitwise the one that problem's own launch in
 * the same variant gives.  With more trajectories than CTAs the graph first
 * sorts all of them, longest first, by the cost score of qram_run_pruned
 * (comparable across problems), in memory allocated and freed inside the
 * graph.
 *   sims: 1 .. 16 simulators on one device, each with a damping-rate bound
 *         (qram_set_gamma_bound, else QRAM_E_STATE) and no depolarizing
 *         faults (else QRAM_E_ARG);
 *   threads: the launch variant for all problems (128, 256 or 512; 0 = that
 *         of sims[0]).  Each simulator is switched to it (qram_set_variant,
 *         which invalidates that simulator's graphs) and its scratch sized;
 *         the dynamic shared memory is the largest problem's.
 * The pointers and counts are bound when the batch is created.
 * qram_batch_launch replays the graph on the stream of sims[0]; work of the
 * other simulators' streams must be ordered before it by the caller.
 * qram_batch_grid returns the number of CTAs of the launch. */
typedef struct qram_batch qram_batch_t;
int qram_batch_create(qram_sim_t *const *sims, uint32_t nsims, int mode, int threads, const uint64_t *traj0,
                      const uint32_t *ntraj, const double *const *gamma, qram_result_t *const *out,
                      qram_batch_t **batch);
int qram_batch_launch(qram_batch_t *batch);
int qram_batch_grid(const qram_batch_t *batch);
void qram_batch_destroy(qram_batch_t *batch);

/* Launch variant: threads per CTA of the trajectory kernel (128, 256, 512
 * or 1024; default 256).  128-512 are the throughput variants (several CTAs,
 * i.e. trajectories, per SM; qram_autotune picks among them).  1024 runs one
 * trajectory per SM with every thread on it: a launch takes about as long as
 * its slowest trajectory, so a small query (few trajectories per SM) finishes
 * sooner, while throughput on large launches is lower.  Results do not
 * depend on the variant except through the order of floating-point block
 * reductions (rounding).  qram_get_variant returns the current one. */
int qram_set_variant(qram_sim_t *sim, int threads);
int qram_get_variant(const qram_sim_t *sim);

/* Autotuner: times one launch of each variant on ntraj trajectories (from
 * traj0) at damping rate gamma in the given mode (0 pruned, 1 full) and
 * keeps the fastest; *best_threads and *best_ms (may be NULL) receive the
 * choice and its time.  Blocks until done; allocates its probe buffers. */
int qram_autotune(qram_sim_t *sim, int mode, double gamma, uint32_t ntraj, uint64_t traj0, int *best_threads,
                  float *best_ms);

/* Trajectory-averaged fidelity (Sec. VI.A: the ensemble mean over sampled
 * noise histories that App. C compares with the density-matrix F_rho) and
 * its Monte Carlo standard error (Fig. 2 error bars: standard error of the
 * mean over trajectories), of results[0 .. ntraj).fidelity (device array).
 * Reduced on the device by one CTA in a fixed order (deterministic); the
 * variance is the unbiased sample variance.  Blocks until the two host
 * doubles are written.  QRAM_E_ARG for null pointers; ntraj = 0 gives 0, 0. */
int qram_fidelity(qram_sim_t *sim, const qram_result_t *results, uint32_t ntraj, double *mean,
                  double *stderr_out);

/* Final normalised state of one trajectory (the exactness check of Sec. VI.A:
 * the pruned and full end states compared amplitude by amplitude): every
 * explicitly evolved component after the second Hadamard wall plus, in
 * pruned mode, the branches held in closed form.  Pruned mode runs the same
 * lazy form as qram_run_pruned: while no jump has fired every branch is in
 * closed form (Prop. 1, Theorem 2), so a jump-free trajectory is emitted
 * entirely from the closed forms; after a jump only the materialised
 * configurations survive (the others are annihilated by K_J).  gamma must be
 * in [0, gamma_lim) (see qram_run_pruned), else QRAM_E_ARG.  Host outputs, capacity cap entries:
 * addr[c], bus[c], config_hash[c] (64-bit hash of the sorted excited-site
 * list, 0 for the ground configuration), re[c], im[c]; *count receives the
 * number of entries (QRAM_E_CAP if it exceeds cap).  mode: 0 pruned, 1 full.
 * Blocks until done. */
int qram_dump_state(qram_sim_t *sim, int mode, uint64_t traj, double gamma, uint32_t cap,
                    uint32_t *addr, uint32_t *bus, uint64_t *config_hash, double *re, double *im,
                    uint32_t *count);

/* Depolarizing faults on top of the amplitude damping (Sec. II.B; App. A;
 * the paper's benchmark setting eps = gamma): every (slice, site) pair of the
 * tree carries, with probability eps, one of the non-identity Pauli
 * operators Z, X, XZ (qubit) or the eight Weyl operators X^a Z^b (qutrit),
 * uniformly, applied after the slice's gates and before its damping layer.
 * Events are drawn on their own fault stream (stream 4, operator words on
 * stream 5; see "Random numbers") and mark bad(v) like damping candidates.
 * eps_equals_gamma != 0 ignores eps and takes each trajectory's damping rate.
 * With eps > 0 every branch is evolved explicitly in both modes (faults on
 * idle sites reach the good branches, which the closed forms of the damping
 * path do not describe).  0 <= eps < 1, else QRAM_E_ARG.  Default 0. */
int qram_set_depolarizing(qram_sim_t *sim, double eps, int eps_equals_gamma);

/* Noise channel of the per-slice layer (default QRAM_CHANNEL_DAMPING, the
 * amplitude damping of Eqs. (5)-(6)).  QRAM_CHANNEL_DEPHASING is the
 * dephasing channel that the outlook (Sec. VII) names as a further channel
 * with a diagonal no-jump operator: phase damping of strength gamma with the
 * same no-jump operator K0 = diag(1, a) (qutrit diag(1, a, a)) and the jump
 * sqrt(gamma)|1><1| (qutrit sqrt(gamma)|L><L|, sqrt(gamma)|R><R|).  Its
 * K_J^dagger K_J is the damping one, so the candidate sampling, the marking,
 * the joint draw of Sec. IV.D and the good-branch closed forms (Prop. 1,
 * Theorem 2) are unchanged; a fired jump projects onto the components that
 * hold its sites excited and leaves their configuration as it is.
 * QRAM_CHANNEL_HEATING is the outlook's heating channel: the diagonal
 * no-jump operator K0 = diag(a, 1, 1) on {W, L, R} (qubit diag(a, 1)) with
 * the jumps sqrt(gamma/2)|L><W| and sqrt(gamma/2)|R><W| (qubit
 * sqrt(gamma)|1><0|).  The joint draw runs over the candidate sites a
 * component holds at the ground level, each with a target level drawn with
 * the candidate (qutrit: bit 0 of word 0 of counter (site, slice | 6 << 24,
 * traj_lo, traj_hi); 0 -> L, 1 -> R); a fired J raises its sites.  Heating
 * jumps reach idle sites of every branch, so with heating both modes evolve
 * every branch (as with depolarizing faults, which cannot be combined with
 * it: QRAM_E_STATE).  Applies to both modes and to qram_dump_state;
 * QRAM_E_ARG for another value. */
int qram_set_channel(qram_sim_t *sim, int channel);

/* Low-weight truncation of the predicted good branches in qram_dump_state
 * (Sec. V, cost discussion after Eq. (26)): each good branch ends in a
 * superposition over all 2^k output words whose amplitude falls by
 * beta/alpha = O(n gamma) per unit of Hamming distance from the ideal word
 * (Eq. (13)); with w_max >= 0 only the words within distance w_max are
 * emitted, the dropped amplitudes being O((n gamma)^(w_max + 1)).
 * w_max = -1 (the default) emits all 2^k words.  Qubit encoding only (the
 * qutrit good branch is a single word); returns QRAM_E_ARG for w_max < -1. */
int qram_set_dump_weight(qram_sim_t *sim, int w_max);

/* Waits for the simulator's stream; returns QRAM_E_CUDA on an asynchronous
 * CUDA error, else QRAM_OK. */
int qram_sync(qram_sim_t *sim);

/* Number of kernel launches issued by this simulator since creation. */
uint64_t qram_launch_count(const qram_sim_t *sim);

/* Work done by this simulator's trajectory launches since creation or the
 * last reset.  No counterpart in the paper: instrumentation for the
 * roofline of the trajectory kernel, and evidence of which evolution forms
 * a launch took.  out (host, 8 entries):
 *   out[0] fault-stream draws (one 64-bit word per geometric gap),
 *   out[1] explicit component-slices (gate slices applied to explicit
 *          components, pruned and full mode),
 *   out[2] branch-epochs of the closed-form weights before the first jump
 *          (nonzero only when the lazy pruned form ran),
 *   out[3] component-epochs of the explicit passes,
 *   out[4] component-slices on the path words of a component with two paths
 *          (a misaligned router sent items off its address path),
 *   out[5] component-slices through the register generic form (path B or
 *          off-path items, at most 8 sites off the address path),
 *   out[6] component-slices through the memory generic form (sorted site
 *          list, up to 32 off-path sites),
 *   out[7] component-epochs that began with off-path items.
 * Each trajectory adds its counts when it finishes.  Waits for the
 * simulator's stream; reset != 0 zeroes the counters afterwards.  Returns
 * QRAM_E_ARG for null pointers, QRAM_E_CUDA on a CUDA error. */
int qram_work_counters(qram_sim_t *sim, uint64_t *out, int reset);

/* ---------------------------------------------------------------------------
 * Serving loop (continuous batching; no paper counterpart, the paper runs
 * one query at a time).  A server owns one device.  Requests are queued by
 * qram_server_submit (non-blocking, inputs copied) and admitted by a native
 * scheduler thread while their estimated device memory fits the budget and
 * fewer than max_active requests run; each admitted request gets its own
 * simulator, stream and share of the SMs, so requests that arrive while
 * others run are admitted as memory frees up and their kernels overlap on
 * the device.  Every trajectory is a pure function of (seed, index, gamma),
 * so a request's results do not depend on what else runs.
 * ------------------------------------------------------------------------- */
typedef struct qram_server qram_server_t;

typedef struct {
    qram_problem_t problem;    /* copied at submit */
    uint64_t traj0;            /* first trajectory index */
    uint32_t ntraj;            /* >= 1 */
    const double *gamma;       /* host, ntraj damping rates in [0, gamma_lim) (copied) */
    int32_t mode;              /* 0 pruned, 1 full */
} qram_request_t;

typedef struct {
    uint64_t id;
    int32_t status;            /* QRAM_OK, a QRAM_E_* code, or QRAM_E_STATE if cancelled */
    uint32_t ntraj;
    double mean_fidelity, stderr_fidelity;   /* qram_fidelity over the request */
    double t_submit, t_admit, t_finish;      /* seconds on the server's steady clock */
    uint64_t device_bytes;     /* device memory the request held */
} qram_completion_t;

/* Create a server on `device` with a device-memory budget in bytes and at
 * most max_active concurrently running requests (>= 1). */
int qram_server_create(size_t mem_budget, int device, uint32_t max_active, qram_server_t **out);

/* Queue a request; *id receives its identifier.  QRAM_E_ARG for a malformed
 * request (same checks as qram_sim_create, a gamma outside [0, gamma_lim)
 * of qram_run_pruned), QRAM_E_OOM
 * if it could never fit the budget, QRAM_E_BUSY if 65536 requests wait. */
int qram_server_submit(qram_server_t *srv, const qram_request_t *req, uint64_t *id);

/* Device bytes the server would reserve for this request (its admission
 * size); QRAM_E_ARG for a malformed request. */
int qram_server_estimate(qram_server_t *srv, const qram_request_t *req, size_t *bytes);

/* Copy up to `max` completions (oldest first) into out; *count receives the
 * number copied.  Non-blocking. */
int qram_server_poll(qram_server_t *srv, qram_completion_t *out, uint32_t max, uint32_t *count);

/* Per-trajectory results of a completed request (host array of cap
 * entries); releases them.  QRAM_E_STATE if the id is unknown or pending. */
int qram_server_results(qram_server_t *srv, uint64_t id, qram_result_t *out, uint32_t cap);

/* Cancel a request: a queued one is dropped, a running one stops taking new
 * trajectories (the trajectories in flight finish); it completes with status
 * QRAM_E_STATE.  QRAM_E_STATE if the id is unknown or already complete. */
int qram_server_cancel(qram_server_t *srv, uint64_t id);

/* Wait (bounded by timeout_s) until no request is queued or running;
 * QRAM_E_TIMEOUT if the time ran out. */
int qram_server_drain(qram_server_t *srv, double timeout_s);

/* Stop the scheduler (running requests finish first) and free everything. */
void qram_server_destroy(qram_server_t *srv);

/* Allocation-free run (no counterpart in the paper; the paper's simulator
 * is a CPU program).  For callers that must not allocate device memory at
 * run time: a host with a fixed device-memory plan made at start-up, code
 * that runs inside another framework's memory pool and may not go around
 * it, or a process whose device memory is already handed out.  Runs the same
 * kernel as qram_run_pruned (mode 0) or qram_run_full (mode 1) on one
 * problem held entirely in caller-owned DEVICE memory:
 *   memory[2^n], addr[D], bus[D], amp_re[D], amp_im[D]  (as in qram_problem_t)
 *   gamma[ntraj] in [0, gamma_lim), out[ntraj]  (as in qram_run_pruned)
 * gamma_max (host) bounds the damping rates (sizes the candidate scratch; a
 * trajectory above it that overflows is reported QRAM_E_CAP).  The inputs
 * are validated on the device; invalid ones make every trajectory report
 * QRAM_E_ARG.  Stream-ordered on cuda_stream (a cudaStream_t, may be NULL)
 * of the current device; returns once enqueued.
 *
 * Scratch: one file-scope device array of 32 MiB per GPU that loads the
 * library, held until the process exits.  The call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  Problems whose
 * scratch for one CTA exceeds the array are rejected with QRAM_E_TOOBIG;
 * smaller ones use as many CTAs as fit.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress): make that first call
 * before any stream capture.  Every call shares the array and it keeps the
 * last call's contents (the call resets what must start at zero itself), so
 * calls that overlap on the GPU (different streams or devices' contexts
 * sharing a device) race: order them on one stream. */
int qram_run_static(int mode, int32_t encoding, int32_t n, int32_t k, int32_t num_branches,
                    const uint8_t *memory, const uint32_t *addr, const uint32_t *bus,
                    const double *amp_re, const double *amp_im, uint64_t seed, uint64_t traj0,
                    uint32_t ntraj, const double *gamma, double gamma_max, qram_result_t *out,
                    void *cuda_stream);
/* (qram_run_static: gamma_max must be below gamma_lim of qram_run_pruned,
 * else QRAM_E_ARG; a trajectory whose own rate reaches gamma_lim reports
 * QRAM_E_ARG.  The static array's device address is cached per device and
 * per CUDA context: after a device reset, or under another context, the
 * next call looks it up again.) */

/* ---------------------------------------------------------------------------
 * Roofline denominators (no paper counterpart: a measurement utility).
 * Measures on `device` the throughput of FP64 fused multiply-adds
 * (*fp64_flops, FLOP/s at 2 per FMA) and of 32-bit integer add and logic
 * instructions (*int32_ops, ops/s), with kernels of eight independent
 * dependency chains per thread on every SM; best of five launches after one
 * untimed.  Synchronous; allocates and frees a small device buffer.  Returns
 * QRAM_E_ARG for null pointers, QRAM_E_CUDA on a CUDA error.
 * ------------------------------------------------------------------------- */
int qram_measure_peaks(int device, double *fp64_flops, double *int32_ops);

/* Static message for a QRAM_* code. */
const char *qram_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* QRAM_SIM_H */
