// qram_internal.h -- launch parameters shared by the host API and the kernels
// of the sm_103a trajectory simulator.  Not part of the C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qram_sim.h"

namespace qram {

constexpr int kMaxN = 14;
constexpr int kMaxK = 8;
constexpr int kMaxT = 6 * kMaxN + 2 * kMaxK;   // 100
constexpr int kXcap = 32;                      // off-path excitations per component
constexpr int kMaxJ = 64;                      // elements of one joint outcome J
// fault stream: (slice, site) pairs are cut into blocks of kGapBlock, and the
// geometric gaps inside a block are at most 2^kGapBits - 1
constexpr uint32_t kGapBlock = 2048;
constexpr int kGapBits = 13;
// Damping exponents are bounded by (2n+k)(T-1) (at most 2n+k excited sites
// per slice); histograms over them need (2n+k)(T-1)+1 <= 3565 bins.
constexpr int kHistMax = 3584;
// Amplitudes are kept unnormalised as a^e (a = sqrt(1 - gamma)), so the
// weights a^(2e) <= (1 - gamma)^((2n+k)(T-1)) must stay in the normal FP64
// range with room for the input weights (>= 2^-22): (2n+k)(T-1) (-ln(1 - gamma))
// is kept below this budget (ln DBL_MIN = -708.4).
constexpr double kLnBudget = 650.0;

enum Mode : int { kPruned = 0, kFull = 1, kSampleOnly = 2 };

// Gates of one time slice (Sec. II.A; App. C).  All act on disjoint slots.
struct SliceOps {
    int8_t load;     // address bit routed at layer `load` is copied into / out of d_0, -1: none
    int8_t bus;      // bus qubit swapped with d_0, -1: none
    int8_t fetch;    // data qubit fetched at the leaf layer, -1: none
    int8_t pad;
    uint32_t iswap;  // bit L: router/data swap on every node of layer L
    uint32_t cswap;  // bit L: controlled swap between layers L and L+1
    uint32_t iswap2; // iswap with bit L moved to bit 2L (path-word layout)
    uint32_t cswap2; // cswap with bit L moved to bit 2L
};

// Per-CTA-slot scratch (device), sized at launch for the worst case.
struct Scratch {
    uint32_t *cand;      // [slots][cand_cap]  packed (slice << 16) | site
    uint32_t *pev;       // [slots][cand_cap]  depolarizing events (slice << 18) | (operator << 15) | site
    uint32_t *wseg;      // [slots][nwarps][seg_cap] per-warp candidate segments
    uint32_t *expl;      // [slots][D] explicit input columns
    // [slots][ecap] packed components, one 16-byte load/store each:
    //   x = path word (bit 2L router, 2L+1 data slot of the path node at layer L)
    //   y = level-R bits of the path word (qutrit)
    //   z = K0 exponent (bits 0-15) | bus word (16-23) | sign (24) | off-path count (25-30)
    //   w = input column (bits 0-13) | address (bits 14-27)
    uint4 *cs;
    uint16_t *exc;       // [slots][ecap][kXcap] off-path sites (site << 1 | isR)
    uint32_t *selk;      // [slots][nwarps][selseg] components with a non-empty mask: first code | size << 16
    double *selw;        // [slots][nwarps][selseg] their weights
    uint32_t *pfr;       // [slots][ecap][8] product-form components: one record per data qubit
    uint32_t cand_cap, seg_cap, ecap, selseg;
};

// Noiseless orbit of the items through the path-word positions.  Items:
// 0 = none, 1 + l = the address bit routed at layer l, 1 + n + t = data
// qubit t.  On a noiseless orbit every gate moves items between positions
// independently of their values (a router holds its address bit before any
// item crosses it), so one table serves every (address, data) pair.
struct Orbit {
    int8_t item[kMaxT][2 * kMaxN];   // item at path-word position b after the gates of slice s
    uint32_t occ[kMaxT];             // positions holding an item
    uint8_t bus[kMaxT];              // bus slots holding their data qubit
    uint8_t fetched[kMaxT];          // data qubits already fetched
    int8_t dpos[kMaxT][kMaxK];       // path-word position of data qubit t after slice s, -1 in the bus
    int ok;                          // 0: the schedule breaks the assumption (no lazy branches)
};

struct DumpOut {
    uint32_t *col;       // [cap] explicit components at the end
    uint32_t *bus;
    uint64_t *hash;
    double *re, *im;
    uint32_t cap;
    uint32_t *count;
    double *scal;        // [4]: W, jump fired, every branch explicit (depolarizing), lazy form
};

struct Params {
    int enc, n, k, T, D, nodes, M, nthreads;
    const uint8_t *mem;
    const uint32_t *addr, *bus;
    const double *amp_re, *amp_im;
    uint64_t seed;
    uint64_t traj0;
    uint32_t ntraj;
    const double *gamma;
    int mode;
    const uint32_t *hist_cand, *hist_off;
    uint32_t nhist;
    qram_result_t *out;
    // sample-only outputs
    uint32_t *o_cand, *o_ncand, *o_badbits, *o_bad;
    int32_t *o_ref;
    uint32_t o_cap;
    Scratch scr;
    uint32_t *work;       // work-stealing counter
    DumpOut dump;
    int dump_mode;
    int dump_wmax;                 // good branches in the dump: output words within this Hamming distance (-1: all)
    const uint32_t *input_error;   // if non-null and nonzero at run time: every trajectory is QRAM_E_ARG
    const double *w2u;             // device scalar: |c|^2 (times 2^-k for qubits) when every column shares it, else 0
    const uint64_t *traj0_dev;     // if non-null, the first trajectory index is read here (graph replays)
    const uint32_t *perm;          // if non-null: the w-th trajectory handed out is perm[w] (see launch_order)
    const uint32_t *col_of;        // qubit input over every address (D = 2^n): column of each address, else null
    double eps;                    // depolarizing strength per (slice, site)
    int eps_gamma;                 // nonzero: the strength of each trajectory is its damping rate
    unsigned long long *ctr;       // if non-null: 8 work counters (see qram_work_counters), added once per trajectory
    int hist_pad;                  // bins per exponent histogram (dynamic shared memory: 3 of them)
    double gamma_lim;              // damping rates at or above this are rejected per trajectory (QRAM_E_ARG)
    int channel;                   // QRAM_CHANNEL_DAMPING or QRAM_CHANNEL_DEPHASING (the jump keeps its sites)
    SliceOps ops[kMaxT];
    uint32_t occ2[kMaxT];  // per slice: path-word positions any noiseless orbit can hold excited
    Orbit orbit;
};

// One persistent launch over several problems (different encodings, n, k):
// the work-stealing counter runs over the concatenated trajectory ranges
// [start[p], start[p + 1]) of problems p = 0 .. nprob - 1, whose Params sit
// in device memory.
constexpr int kMaxBatch = 16;
struct MultiParams {
    const Params *probs;          // device, nprob entries
    uint32_t *work;               // work-stealing counter over all trajectories
    uint32_t nprob;
    uint32_t dyn_words;           // dynamic shared memory (32-bit words): the largest problem's
    const uint32_t *perm;         // if non-null: the w-th trajectory handed out is perm[w] (launch_order_multi)
    uint32_t start[kMaxBatch + 1];
};

cudaError_t launch_trajectories(const Params &p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_trajectories_multi(const MultiParams &mp, int grid, int block, size_t smem, cudaStream_t s);
int kernel_blocks_per_sm_multi(int threads, size_t dyn);
// Launch order, longest first: score = a cost score per trajectory (its
// damping candidates, regenerated, weighted by the branches a jump there
// would leave explicit), then perm = the indices 0 .. ntraj-1 sorted into
// buckets of descending score (rejected rates last), any order inside a
// bucket.  perm and score: device, ntraj entries each.
constexpr int kOrderBuckets = 64;
cudaError_t launch_order(const Params &p, uint32_t ntraj, uint32_t *perm, float *score, cudaStream_t s);
// The same over the concatenated ranges of a mixed launch (mp.probs on the
// device, mp.start and mp.nprob set); nmax, tmax: the largest n and T.
cudaError_t launch_order_multi(const MultiParams &mp, int nmax, int tmax, uint32_t *perm, float *score,
                               cudaStream_t s);
cudaError_t launch_fidelity(const qram_result_t *res, uint32_t ntraj, double *out2, cudaStream_t s);
cudaError_t launch_uniform_weight(const double *re, const double *im, int D, int qubit_k, double *out, cudaStream_t s);
cudaError_t launch_dump_finalize(const Params &p, uint32_t n_in, uint32_t *out_n, uint32_t cap,
                                 uint32_t *o_addr, uint32_t *o_bus, uint64_t *o_hash, double *o_re,
                                 double *o_im, cudaStream_t s);
// host-side helpers shared by the API and the serving loop
// largest damping rate (exclusive) whose unnormalised weights stay in range (kLnBudget)
double gamma_limit(int n, int k);
size_t estimate_sim_bytes(int enc, int n, int k, int D, int slots, double gmax, int threads);
int build_ops(int n, int k, SliceOps *ops);
// occ2[s] = (layer, slot) positions, as path-word bits, that an item can
// occupy after the gates of slice s in a noiseless orbit
void build_occupancy(int n, int k, const SliceOps *ops, uint32_t *occ2);
// the item table of the noiseless orbit (see Orbit)
void build_orbit(int n, int k, const SliceOps *ops, Orbit *orb);
// lays out the per-slot scratch of `slots` CTAs at `base` (may be null: size only); returns bytes
size_t carve_scratch(int enc, int n, int k, int D, int slots, double gmax, int threads, void *base, Scratch *scr);
int resident_slots_per_device(int device, int threads, size_t dyn);

int kernel_threads();                                   // default variant
bool valid_threads(int threads);                        // 128, 256, 512 or 1024
int kernel_blocks_per_sm(int threads, size_t dyn);      // resident CTAs per SM of a variant
int hist_pad(int n, int k);
size_t dyn_smem_bytes(int n, int k, int threads = 512);   // bytes for a variant (at most 512 threads: the same)

}  // namespace qram
