// qram_api.cu -- host implementation of the C ABI declared in include/qram_sim.h.
//
// Owns the device copies of a problem, builds the slice gate table of the
// time-sliced bucket-brigade schedule (Sec. II.A, Eqs. (2)-(4); App. C gate
// list), sizes the per-CTA scratch and launches the kernels of
// qram_kernels.cu.  No CPU computation of the method happens here.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "qram_internal.h"

using namespace qram;

struct qram_sim {
    int device = 0;
    cudaStream_t stream = nullptr;
    int enc = 0, n = 0, k = 0, D = 0, T = 0;
    uint64_t seed = 0;
    uint8_t *d_mem = nullptr;
    uint32_t *d_addr = nullptr, *d_bus = nullptr;
    double *d_re = nullptr, *d_im = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    Scratch scr{};
    int slots = 0;
    uint32_t *d_work = nullptr;
    double *d_fid2 = nullptr;
    double *d_gmax = nullptr;
    double *d_w2u = nullptr;
    uint32_t *d_colof = nullptr;    // complete qubit input: column of each address
    const uint32_t *hist_cand = nullptr, *hist_off = nullptr;
    uint32_t nhist = 0;
    SliceOps ops[kMaxT]{};
    uint32_t occ2[kMaxT]{};
    Orbit orbit{};
    uint64_t launches = 0;
    int sms = 0, blocks_per_sm = 0;
    int threads = 256;          // launch variant (threads per CTA)
    size_t dyn = 0;             // dynamic shared memory per CTA
    int scr_threads = 0;        // variant the scratch was laid out for
    double gamma_bound = 0.0;
    int dump_wmax = -1;         // low-weight truncation of the dumped good branches
    double eps = 0.0;           // depolarizing strength
    int eps_gamma = 0;          // the strength of each trajectory is its damping rate
    int channel = QRAM_CHANNEL_DAMPING;
};

namespace {

bool ok(cudaError_t e) { return e == cudaSuccess; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// Slot bookkeeping for the disjointness check of one slice: tree sites,
// then address bits, then bus qubits.
struct SlotUse {
    std::vector<uint8_t> used;
    bool take(size_t s) { if (used[s]) return false; used[s] = 1; return true; }
};

// Schedule of Sec. II.A: address bit l (routed at layer l) enters d_0 at
// 2l+1, walks down one layer per slice, settles in the router of layer l at
// 3l+2 and returns along the mirror image s -> T-s; data qubit t enters at
// 2n+2t+1, is fetched at the leaf layer at 3n+2t+1 and leaves at 4n+2t+1.
int build_ops_impl(int n, int k, SliceOps *ops) {
    const int T = 6 * n + 2 * k;
    for (int s = 0; s < kMaxT; ++s) { ops[s].load = -1; ops[s].bus = -1; ops[s].fetch = -1; ops[s].pad = 0; ops[s].iswap = 0; ops[s].cswap = 0; }
    auto set8 = [](int8_t &f, int v) { if (f >= 0 && f != v) return false; f = (int8_t)v; return true; };
    for (int l = 0; l < n; ++l) {
        if (!set8(ops[2 * l + 1].load, l) || !set8(ops[T - 2 * l - 1].load, l)) return QRAM_E_ARG;
        for (int m = 1; m <= l; ++m) {
            ops[2 * l + 1 + m].cswap |= 1u << (m - 1);
            ops[T - 2 * l - 1 - m].cswap |= 1u << (m - 1);
        }
        ops[3 * l + 2].iswap |= 1u << l;
        ops[T - 3 * l - 2].iswap |= 1u << l;
    }
    for (int t = 0; t < k; ++t) {
        if (!set8(ops[2 * n + 2 * t + 1].bus, t) || !set8(ops[4 * n + 2 * t + 1].bus, t)) return QRAM_E_ARG;
        for (int m = 1; m <= n - 1; ++m) {
            ops[2 * n + 2 * t + 1 + m].cswap |= 1u << (m - 1);
            ops[3 * n + 2 * t + 1 + m].cswap |= 1u << (n - 1 - m);
        }
        if (!set8(ops[3 * n + 2 * t + 1].fetch, t)) return QRAM_E_ARG;
    }
    for (int s = 0; s < kMaxT; ++s) {
        uint32_t a = 0, b = 0;
        for (int L = 0; L < 16; ++L) {
            if ((ops[s].iswap >> L) & 1u) a |= 1u << (2 * L);
            if ((ops[s].cswap >> L) & 1u) b |= 1u << (2 * L);
        }
        ops[s].iswap2 = a;
        ops[s].cswap2 = b;
    }
    // every gate of a slice must act on its own slots (controls included)
    const size_t M = 2 * ((size_t(1) << n) - 1);
    SlotUse U;
    for (int s = 1; s < T; ++s) {
        U.used.assign(M + n + k, 0);
        const SliceOps &o = ops[s];
        if (o.load >= 0 && o.bus >= 0) return QRAM_E_ARG;      // both need d_0
        if (o.load >= 0 && (!U.take(1) || !U.take(M + o.load))) return QRAM_E_ARG;
        if (o.bus >= 0 && (!U.take(1) || !U.take(M + n + o.bus))) return QRAM_E_ARG;
        for (int L = 0; L < n; ++L) {
            const size_t lo = (size_t(1) << L) - 1, hi = (size_t(2) << L) - 1;
            if ((o.iswap >> L) & 1u)
                for (size_t v = lo; v < hi; ++v) if (!U.take(2 * v) || !U.take(2 * v + 1)) return QRAM_E_ARG;
            if ((o.cswap >> L) & 1u) {
                if (L + 1 >= n) return QRAM_E_ARG;
                for (size_t v = lo; v < hi; ++v)
                    if (!U.take(2 * v) || !U.take(2 * v + 1) || !U.take(2 * (2 * v + 1) + 1) || !U.take(2 * (2 * v + 2) + 1))
                        return QRAM_E_ARG;
            }
        }
        if (o.fetch >= 0)
            for (size_t v = (size_t(1) << (n - 1)) - 1; v < (size_t(1) << n) - 1; ++v)
                if (!U.take(2 * v) || !U.take(2 * v + 1)) return QRAM_E_ARG;
    }
    return QRAM_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// per-slot candidate capacities for a damping-rate bound gmax: mean + 12 sigma
void cand_caps(int n, int k, double gmax, int threads, uint32_t *cand_cap, uint32_t *seg_cap) {
    const int NWARP = threads / 32;
    // fault sites: (slice, site) pairs; a warp takes a contiguous run of
    // blocks of kGapBlock pairs
    const double sites = (double)(6 * n + 2 * k - 1) * 2.0 * (double)((1u << n) - 1);
    const double nblk = std::ceil(sites / kGapBlock);
    const double per = std::min(sites, std::ceil(nblk / NWARP) * kGapBlock);
    auto cap = [&](double m) {
        const double p = std::min(1.0, std::max(gmax, 0.0));
        const double mean = m * p, sd = std::sqrt(m * p * (1.0 - p) + 1.0);
        double c = mean + 12.0 * sd + 64.0;
        c = std::min(c, m + 64.0);
        return (uint32_t)(std::ceil(c / 32.0) * 32.0);
    };
    *cand_cap = cap(sites);
    *seg_cap = cap(per);
}

struct Layout {
    size_t o_cand, o_pev, o_seg, o_expl, o_cs, o_exc, o_selk, o_selw, o_pfr, total;
    uint32_t cc, sc, ecap, selseg;
};

Layout scratch_layout(int enc, int n, int k, int D, size_t slots, double gmax, int threads) {
    Layout L;
    cand_caps(n, k, gmax, threads, &L.cc, &L.sc);
    L.ecap = (uint32_t)D << (enc == QRAM_QUBIT ? k : 0);
    const int NWARP = threads / 32;
    size_t off = 0;
    L.o_cand = off; off = align_up(off + slots * L.cc * 4);
    L.o_pev = off; off = align_up(off + slots * L.cc * 4);
    L.o_seg = off; off = align_up(off + slots * NWARP * (size_t)L.sc * 4);
    L.o_expl = off; off = align_up(off + slots * (size_t)D * 4);
    L.o_cs = off; off = align_up(off + slots * (size_t)L.ecap * 16);
    L.o_exc = off; off = align_up(off + slots * (size_t)L.ecap * kXcap * 2);
    // per-warp segments: warp w sees at most ceil(ecap / threads) * 32 components
    // (also when each thread of a warp materialises all configurations of one branch)
    const size_t per_comp = ((size_t)L.ecap + threads - 1) / threads * 32;
    const size_t per_branch = ((size_t)D + threads - 1) / threads * 32 * ((size_t)L.ecap / (size_t)std::max(D, 1));
    L.selseg = (uint32_t)std::max(per_comp, per_branch);
    L.o_selk = off; off = align_up(off + slots * (size_t)NWARP * L.selseg * 4);
    L.o_selw = off; off = align_up(off + slots * (size_t)NWARP * L.selseg * 8);
    // product-form records: qubit, k >= 2 (one per component, 8 words)
    L.o_pfr = off; off = align_up(off + ((enc == QRAM_QUBIT && k >= 2) ? slots * (size_t)L.ecap * 32 : 0));
    L.total = off;
    return L;
}

int ensure_scratch(qram_sim *S, double gmax) {
    gmax = std::max(gmax, S->eps);                     // depolarizing events share the candidate capacity
    const Layout L = scratch_layout(S->enc, S->n, S->k, S->D, (size_t)S->slots, gmax, S->threads);
    if (S->scratch && S->scr_threads == S->threads && S->scr.cand_cap >= L.cc && S->scr.seg_cap >= L.sc &&
        S->scr.ecap >= L.ecap)
        return QRAM_OK;
    // stream-ordered: no device-wide synchronisation, so other work keeps running
    if (S->scratch) { cudaFreeAsync(S->scratch, S->stream); S->scratch = nullptr; }
    void *p = nullptr;
    if (!ok(cudaMallocAsync(&p, L.total, S->stream))) { cudaGetLastError(); return QRAM_E_OOM; }
    char *b = (char *)p;
    S->scratch = p;
    S->scratch_bytes = L.total;
    S->scr.cand = (uint32_t *)(b + L.o_cand);
    S->scr.pev = (uint32_t *)(b + L.o_pev);
    S->scr.wseg = (uint32_t *)(b + L.o_seg);
    S->scr.expl = (uint32_t *)(b + L.o_expl);
    S->scr.cs = (uint4 *)(b + L.o_cs);
    S->scr.exc = (uint16_t *)(b + L.o_exc);
    S->scr.selk = (uint32_t *)(b + L.o_selk);
    S->scr.selw = (double *)(b + L.o_selw);
    S->scr.pfr = (uint32_t *)(b + L.o_pfr);
    S->scr.selseg = L.selseg;
    S->scr.cand_cap = L.cc;
    S->scr.seg_cap = L.sc;
    S->scr.ecap = L.ecap;
    S->scr_threads = S->threads;
    return QRAM_OK;
}

__global__ void gmax_kernel(const double *g, uint32_t n, double *out) {
    __shared__ double m[256];
    double x = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += 256) { const double v = g[i]; if (!(v <= x)) x = v; }
    m[threadIdx.x] = x;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) { const double v = m[threadIdx.x + s]; if (!(v <= m[threadIdx.x])) m[threadIdx.x] = v; }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = m[0];
}

Params base_params(qram_sim *S) {
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.enc = S->enc; P.n = S->n; P.k = S->k; P.T = S->T; P.D = S->D;
    P.nodes = (1 << S->n) - 1; P.M = 2 * P.nodes; P.nthreads = S->threads; P.hist_pad = hist_pad(S->n, S->k);
    P.mem = S->d_mem; P.addr = S->d_addr; P.bus = S->d_bus; P.amp_re = S->d_re; P.amp_im = S->d_im;
    P.seed = S->seed;
    P.hist_cand = S->hist_cand; P.hist_off = S->hist_off; P.nhist = S->nhist;
    P.scr = S->scr;
    P.work = S->d_work;
    P.w2u = S->d_w2u;
    P.col_of = S->d_colof;
    P.eps = S->eps;
    P.eps_gamma = S->eps_gamma;
    P.ctr = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(S->d_work) + 32);
    P.gamma_lim = gamma_limit(S->n, S->k);
    P.channel = S->channel;
    std::memcpy(P.ops, S->ops, sizeof(P.ops));
    std::memcpy(P.occ2, S->occ2, sizeof(P.occ2));
    P.orbit = S->orbit;
    return P;
}

int bound_gamma(qram_sim *S, const double *gamma, uint32_t ntraj, double *gmax) {
    if (S->gamma_bound > 0.0) { *gmax = S->gamma_bound; return QRAM_OK; }
    gmax_kernel<<<1, 256, 0, S->stream>>>(gamma, ntraj, S->d_gmax);
    S->launches++;
    if (!ok(cudaGetLastError())) return QRAM_E_CUDA;
    double g = 0;
    if (!ok(cudaMemcpyAsync(&g, S->d_gmax, sizeof(double), cudaMemcpyDeviceToHost, S->stream))) return QRAM_E_CUDA;
    if (!ok(cudaStreamSynchronize(S->stream))) return QRAM_E_CUDA;
    if (!(g >= 0.0 && g < 1.0)) g = 1.0;           // invalid rates are flagged per trajectory
    *gmax = g;
    return QRAM_OK;
}

// Enqueues one trajectory launch on st.  A pruned or full launch with more
// trajectories than CTAs first scores and sorts its trajectories by expected
// cost, longest first (launch_order), in stream-ordered memory that is freed
// again after the launch (inside a capture: memory nodes of the graph);
// without that memory the trajectories go in index order.  *nk: kernels
// enqueued.
int enqueue(qram_sim *S, Params &P, uint32_t ntraj, int grid, double gmax, cudaStream_t st, int *nk) {
    *nk = 0;
    uint32_t *perm = nullptr;
    if ((P.mode == kPruned || P.mode == kFull) && ntraj > (uint32_t)grid && gmax > 0.0) {
        if (ok(cudaMallocAsync((void **)&perm, (size_t)ntraj * (sizeof(uint32_t) + sizeof(float)), st))) {
            if (!ok(launch_order(P, ntraj, perm, reinterpret_cast<float *>(perm + ntraj), st))) {
                cudaFreeAsync(perm, st);
                return QRAM_E_CUDA;
            }
            P.perm = perm;
            *nk += 2;
        } else {
            cudaGetLastError();
            perm = nullptr;
        }
    }
    int rc = QRAM_OK;
    if (!ok(cudaMemsetAsync(S->d_work, 0, sizeof(uint32_t), st)) ||
        !ok(launch_trajectories(P, grid, S->threads, S->dyn, st)))
        rc = QRAM_E_CUDA;
    else
        ++*nk;
    if (perm) cudaFreeAsync(perm, st);
    P.perm = nullptr;
    return rc;
}

int launch(qram_sim *S, Params &P, uint32_t ntraj, double gmax) {
    const int grid = (int)std::min<uint32_t>((uint32_t)S->slots, std::max<uint32_t>(ntraj, 1u));
    int nk = 0;
    const int rc = enqueue(S, P, ntraj, grid, gmax, S->stream, &nk);
    S->launches += (uint64_t)nk;
    return rc;
}

int run_mode(qram_sim *S, int mode, uint64_t traj0, uint32_t ntraj, const double *gamma, qram_result_t *out) {
    if (!S || !gamma || !out) return QRAM_E_ARG;
    if (ntraj == 0) return QRAM_OK;
    DeviceGuard g(S->device);
    double gmax;
    int rc = bound_gamma(S, gamma, ntraj, &gmax);
    if (rc) return rc;
    if ((rc = ensure_scratch(S, gmax))) return rc;
    Params P = base_params(S);
    P.traj0 = traj0; P.ntraj = ntraj; P.gamma = gamma; P.mode = mode; P.out = out;
    return launch(S, P, ntraj, gmax);
}

}  // namespace

namespace qram {

int build_ops(int n, int k, SliceOps *ops) { return build_ops_impl(n, k, ops); }

double gamma_limit(int n, int k) {
    const double emax = (double)(2 * n + k) * (double)(6 * n + 2 * k - 1);
    return -std::expm1(-kLnBudget / emax);                 // 1 - exp(-budget / emax)
}

// Noiseless orbit with every item excited (all address bits 1, all data bits
// 1): its path word after each slice marks every position an item can hold.
void build_occupancy(int n, int k, const SliceOps *ops, uint32_t *occ2) {
    const int T = 6 * n + 2 * k;
    uint32_t pw = 0, bus = (1u << k) - 1u;
    for (int s = 0; s < kMaxT; ++s) occ2[s] = 0;
    for (int s = 1; s < T; ++s) {
        const SliceOps &o = ops[s];
        if (o.load >= 0) pw ^= 2u;
        if (o.bus >= 0) {
            const uint32_t d0 = (pw >> 1) & 1u, b = (bus >> o.bus) & 1u;
            pw = (pw & ~2u) | (b << 1);
            bus = (bus & ~(1u << o.bus)) | (d0 << o.bus);
        }
        uint32_t t = (pw ^ (pw >> 1)) & o.iswap2;
        pw ^= t | (t << 1);
        t = (pw ^ (pw >> 2)) & (o.cswap2 << 1);
        pw ^= t | (t << 2);
        occ2[s] = pw;
    }
}

void build_orbit(int n, int k, const SliceOps *ops, Orbit *orb) {
    std::memset(orb, 0, sizeof(*orb));
    const int T = 6 * n + 2 * k;
    int8_t pos[2 * kMaxN] = {0}, bus[kMaxK] = {0};
    for (int t = 0; t < k; ++t) bus[t] = (int8_t)(1 + n + t);
    auto is_addr = [&](int it) { return it >= 1 && it <= n; };
    uint32_t fetched = 0;
    bool good = true;
    int in_tree[kMaxN + kMaxK] = {0}, first[kMaxN + kMaxK], last[kMaxN + kMaxK], fetch_at[kMaxK];
    for (int x = 0; x < kMaxN + kMaxK; ++x) { first[x] = -1; last[x] = -1; }
    for (int t = 0; t < kMaxK; ++t) fetch_at[t] = -1;
    for (int s = 1; s < T; ++s) {
        const SliceOps &o = ops[s];
        if (o.load >= 0) {
            const int8_t a = (int8_t)(1 + o.load);
            if (pos[1] == 0) pos[1] = a;
            else if (pos[1] == a) pos[1] = 0;
            else good = false;
        }
        if (o.bus >= 0) {
            if (is_addr(pos[1])) good = false;
            std::swap(pos[1], bus[o.bus]);
            if (bus[o.bus] != 0 && bus[o.bus] != 1 + n + o.bus) good = false;
        }
        for (int L = 0; L < n; ++L)
            if ((o.iswap >> L) & 1u) std::swap(pos[2 * L], pos[2 * L + 1]);
        for (int L = 0; L + 1 < n; ++L) {
            if (!((o.cswap >> L) & 1u)) continue;
            // an item may only cross a router that already holds its address bit
            if ((pos[2 * L + 1] || pos[2 * L + 3]) && !is_addr(pos[2 * L])) good = false;
            std::swap(pos[2 * L + 1], pos[2 * L + 3]);
        }
        if (o.fetch >= 0) {
            if (pos[2 * (n - 1) + 1] != 1 + n + o.fetch || !is_addr(pos[2 * (n - 1)])) good = false;
            fetched |= 1u << o.fetch;
            fetch_at[o.fetch] = s;
        }
        uint32_t occ = 0, bm = 0;
        for (int b = 0; b < 2 * n; ++b) {
            orb->item[s][b] = pos[b];
            if (pos[b]) {
                occ |= 1u << b;
                const int x = pos[b] - 1;
                ++in_tree[x];
                if (first[x] < 0) first[x] = s;
                last[x] = s;
            }
        }
        for (int t = 0; t < kMaxK; ++t) orb->dpos[s][t] = -1;
        for (int b = 0; b < 2 * n; ++b)
            if (pos[b] > n) orb->dpos[s][pos[b] - 1 - n] = (int8_t)b;
        for (int t = 0; t < k; ++t) if (bus[t] == 1 + n + t) bm |= 1u << t;
        orb->occ[s] = occ;
        orb->bus[s] = (uint8_t)bm;
        orb->fetched[s] = (uint8_t)fetched;
    }
    // the kernels take the exposures in closed form: address bit l in the tree
    // during slices [2l+1, T-2l-2], data qubit t during [2n+2t+1, 4n+2t],
    // fetched at 3n+2t+1 (Sec. II.A); the orbit must end with an empty tree
    for (int l = 0; l < n; ++l)
        if (first[l] != 2 * l + 1 || last[l] != T - 2 * l - 2 || in_tree[l] != last[l] - first[l] + 1) good = false;
    for (int t = 0; t < k; ++t) {
        const int x = n + t;
        if (first[x] != 2 * n + 2 * t + 1 || last[x] != 4 * n + 2 * t || in_tree[x] != 2 * n) good = false;
        if (fetch_at[t] != 3 * n + 2 * t + 1) good = false;
    }
    if (orb->occ[T - 1] != 0 || orb->bus[T - 1] != (uint8_t)((1u << k) - 1u)) good = false;
    orb->ok = good ? 1 : 0;
}

size_t carve_scratch(int enc, int n, int k, int D, int slots, double gmax, int threads, void *base, Scratch *scr) {
    const Layout L = scratch_layout(enc, n, k, D, (size_t)slots, gmax, threads);
    if (base) {
        char *b = (char *)base;
        scr->cand = (uint32_t *)(b + L.o_cand);
        scr->pev = (uint32_t *)(b + L.o_pev);
        scr->wseg = (uint32_t *)(b + L.o_seg);
        scr->expl = (uint32_t *)(b + L.o_expl);
        scr->cs = (uint4 *)(b + L.o_cs);
        scr->exc = (uint16_t *)(b + L.o_exc);
        scr->selk = (uint32_t *)(b + L.o_selk);
        scr->selw = (double *)(b + L.o_selw);
        scr->pfr = (uint32_t *)(b + L.o_pfr);
        scr->selseg = L.selseg;
        scr->cand_cap = L.cc;
        scr->seg_cap = L.sc;
        scr->ecap = L.ecap;
    }
    return L.total;
}

size_t estimate_sim_bytes(int enc, int n, int k, int D, int slots, double gmax, int threads) {
    const size_t prob = (size_t(1) << n) + (size_t)D * 24 + 4096;
    return prob + scratch_layout(enc, n, k, D, (size_t)slots, gmax, threads).total;
}

int resident_slots_per_device(int device, int threads, size_t dyn) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return sms * kernel_blocks_per_sm(threads, dyn);
}

}  // namespace qram

extern "C" {

const char *qram_strerror(int code) {
    switch (code) {
    case QRAM_OK: return "ok";
    case QRAM_E_ARG: return "invalid argument";
    case QRAM_E_OOM: return "out of memory";
    case QRAM_E_CUDA: return "CUDA runtime error";
    case QRAM_E_TIMEOUT: return "bounded device wait timed out";
    case QRAM_E_BUSY: return "busy";
    case QRAM_E_CAP: return "per-trajectory capacity exceeded";
    case QRAM_E_STATE: return "invalid state";
    case QRAM_E_TOOBIG: return "problem exceeds the static scratch of the allocation-free entry point";
    default: return "unknown error";
    }
}

int qram_sim_create(const qram_problem_t *p, int device, void *cuda_stream, qram_sim_t **out) {
    if (!p || !out) return QRAM_E_ARG;
    *out = nullptr;
    if (p->encoding != QRAM_QUTRIT && p->encoding != QRAM_QUBIT) return QRAM_E_ARG;
    if (p->n < 1 || p->n > kMaxN || p->k < 1 || p->k > kMaxK || p->k > p->n) return QRAM_E_ARG;
    if (p->sampler_version != QRAM_SAMPLER_VERSION) return QRAM_E_ARG;
    const uint32_t N = 1u << p->n;
    if (p->num_branches < 1 || (uint32_t)p->num_branches > N) return QRAM_E_ARG;
    if (!p->memory || !p->addr || !p->bus || !p->amp_re || !p->amp_im) return QRAM_E_ARG;
    std::vector<uint8_t> seen(N, 0);
    double nrm = 0.0;
    for (int b = 0; b < p->num_branches; ++b) {
        if (p->addr[b] >= N || seen[p->addr[b]]) return QRAM_E_ARG;    // one column per address
        seen[p->addr[b]] = 1;
        if (p->bus[b] >= (1u << p->k)) return QRAM_E_ARG;
        if (!std::isfinite(p->amp_re[b]) || !std::isfinite(p->amp_im[b])) return QRAM_E_ARG;
        nrm += p->amp_re[b] * p->amp_re[b] + p->amp_im[b] * p->amp_im[b];
    }
    if (std::fabs(nrm - 1.0) > 1e-12) return QRAM_E_ARG;
    for (uint32_t i = 0; i < N; ++i) if (p->memory[i] >= (1u << p->k)) return QRAM_E_ARG;

    qram_sim *S = new (std::nothrow) qram_sim();
    if (!S) return QRAM_E_OOM;
    S->device = device;
    S->stream = (cudaStream_t)cuda_stream;
    S->enc = p->encoding; S->n = p->n; S->k = p->k; S->D = p->num_branches; S->T = 6 * p->n + 2 * p->k;
    S->seed = p->seed;
    if (build_ops_impl(S->n, S->k, S->ops) != QRAM_OK) { delete S; return QRAM_E_ARG; }
    build_occupancy(S->n, S->k, S->ops, S->occ2);
    build_orbit(S->n, S->k, S->ops, &S->orbit);
    DeviceGuard g(device);
    int rc = QRAM_OK;
    const size_t D = (size_t)S->D;
    if (!ok(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, device))) { delete S; return QRAM_E_CUDA; }
    S->dyn = dyn_smem_bytes(S->n, S->k);
    S->blocks_per_sm = kernel_blocks_per_sm(S->threads, S->dyn);
    if (S->blocks_per_sm < 1) { delete S; return QRAM_E_CUDA; }
    S->slots = S->sms * S->blocks_per_sm;
    cudaStream_t st = S->stream;
    if (!ok(cudaMallocAsync((void **)&S->d_mem, N, st)) || !ok(cudaMallocAsync((void **)&S->d_addr, D * 4, st)) ||
        !ok(cudaMallocAsync((void **)&S->d_bus, D * 4, st)) || !ok(cudaMallocAsync((void **)&S->d_re, D * 8, st)) ||
        !ok(cudaMallocAsync((void **)&S->d_im, D * 8, st)) || !ok(cudaMallocAsync((void **)&S->d_work, 128, st)) ||
        !ok(cudaMallocAsync((void **)&S->d_fid2, 16, st)) || !ok(cudaMallocAsync((void **)&S->d_gmax, 8, st)) ||
        !ok(cudaMallocAsync((void **)&S->d_w2u, 8, st))) {
        cudaGetLastError();
        qram_sim_destroy(S);
        return QRAM_E_OOM;
    }
    // pageable sources: each copy returns once the host data is staged
    if (!ok(cudaMemcpyAsync(S->d_mem, p->memory, N, cudaMemcpyHostToDevice, st)) ||
        !ok(cudaMemcpyAsync(S->d_addr, p->addr, D * 4, cudaMemcpyHostToDevice, st)) ||
        !ok(cudaMemcpyAsync(S->d_bus, p->bus, D * 4, cudaMemcpyHostToDevice, st)) ||
        !ok(cudaMemcpyAsync(S->d_re, p->amp_re, D * 8, cudaMemcpyHostToDevice, st)) ||
        !ok(cudaMemcpyAsync(S->d_im, p->amp_im, D * 8, cudaMemcpyHostToDevice, st)))
        rc = QRAM_E_CUDA;
    if (!rc && !ok(cudaMemsetAsync(S->d_work, 0, 128, st))) rc = QRAM_E_CUDA;    // counter + 8 work counters at +32
    // every address present (qubit): the closed-form weights factorise over the address bits
    if (!rc && S->enc == QRAM_QUBIT && D == N) {
        std::vector<uint32_t> col(N);
        for (uint32_t b = 0; b < (uint32_t)D; ++b) col[p->addr[b]] = b;
        if (!ok(cudaMallocAsync((void **)&S->d_colof, N * 4, st)) ||
            !ok(cudaMemcpyAsync(S->d_colof, col.data(), N * 4, cudaMemcpyHostToDevice, st)) ||
            !ok(cudaStreamSynchronize(st)))                 // the host vector goes out of scope
            rc = QRAM_E_CUDA;
    }
    if (!rc && !ok(launch_uniform_weight(S->d_re, S->d_im, S->D, S->enc == QRAM_QUBIT ? S->k : 0, S->d_w2u, st)))
        rc = QRAM_E_CUDA;
    if (!rc) S->launches++;
    if (rc) { qram_sim_destroy(S); return rc; }
    *out = S;
    return QRAM_OK;
}

void qram_sim_destroy(qram_sim_t *S) {
    if (!S) return;
    {
        DeviceGuard g(S->device);
        cudaStream_t st = S->stream;
        void *bufs[] = {S->d_mem,  S->d_addr, S->d_bus,  S->d_re,  S->d_im,    S->d_work,
                        S->d_fid2, S->d_gmax, S->d_w2u,  S->d_colof, S->scratch};
        for (void *b : bufs) if (b) cudaFreeAsync(b, st);
        cudaStreamSynchronize(st);
        cudaGetLastError();
    }
    delete S;
}

int qram_sample_faults(qram_sim_t *S, uint64_t traj0, uint32_t ntraj, const double *gamma, uint32_t cap,
                       uint32_t *cand, uint32_t *ncand, uint32_t *bad_bits, uint32_t *bad, int32_t *ref) {
    if (!S || !gamma || !cand || !ncand || !bad_bits || !bad || !ref) return QRAM_E_ARG;
    if (ntraj == 0) return QRAM_OK;
    DeviceGuard g(S->device);
    double gmax;
    int rc = bound_gamma(S, gamma, ntraj, &gmax);
    if (rc) return rc;
    if ((rc = ensure_scratch(S, gmax))) return rc;
    Params P = base_params(S);
    P.traj0 = traj0; P.ntraj = ntraj; P.gamma = gamma; P.mode = kSampleOnly;
    P.o_cand = cand; P.o_ncand = ncand; P.o_badbits = bad_bits; P.o_bad = bad; P.o_ref = ref; P.o_cap = cap;
    return launch(S, P, ntraj, gmax);
}

int qram_run_pruned(qram_sim_t *S, uint64_t traj0, uint32_t ntraj, const double *gamma, qram_result_t *out) {
    return run_mode(S, kPruned, traj0, ntraj, gamma, out);
}

int qram_run_full(qram_sim_t *S, uint64_t traj0, uint32_t ntraj, const double *gamma, qram_result_t *out) {
    return run_mode(S, kFull, traj0, ntraj, gamma, out);
}

int qram_set_fault_history(qram_sim_t *S, uint32_t nhist, const uint32_t *cand, const uint32_t *off) {
    if (!S) return QRAM_E_ARG;
    if (nhist > 0 && (!cand || !off)) return QRAM_E_ARG;
    S->nhist = nhist;
    S->hist_cand = nhist ? cand : nullptr;
    S->hist_off = nhist ? off : nullptr;
    return QRAM_OK;
}

struct qram_graph {
    qram_sim *sim = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nk = 0;                      // kernels per replay
};

int qram_graph_create(qram_sim_t *S, int mode, uint32_t ntraj, const double *gamma, qram_result_t *out,
                      const uint64_t *traj0_dev, qram_graph_t **gout) {
    if (!S || !gamma || !out || !traj0_dev || !gout || ntraj == 0 || (mode != 0 && mode != 1)) return QRAM_E_ARG;
    if (!(S->gamma_bound > 0.0)) return QRAM_E_STATE;              // no host read-back inside a capture
    *gout = nullptr;
    DeviceGuard g(S->device);
    int rc = ensure_scratch(S, S->gamma_bound);
    if (rc) return rc;
    if (S->stream && !ok(cudaStreamSynchronize(S->stream))) return QRAM_E_CUDA;
    cudaStream_t cap = nullptr;
    if (!ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return QRAM_E_CUDA;
    qram_graph *G = new (std::nothrow) qram_graph();
    if (!G) { cudaStreamDestroy(cap); return QRAM_E_OOM; }
    G->sim = S;
    Params P = base_params(S);
    P.ntraj = ntraj; P.gamma = gamma; P.mode = mode == 0 ? kPruned : kFull; P.out = out; P.traj0_dev = traj0_dev;
    const int grid = (int)std::min<uint32_t>((uint32_t)S->slots, ntraj);
    rc = QRAM_OK;
    if (!ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) rc = QRAM_E_CUDA;
    else {
        rc = enqueue(S, P, ntraj, grid, S->gamma_bound, cap, &G->nk);
        cudaGraph_t graph = nullptr;
        if (!ok(cudaStreamEndCapture(cap, &graph))) rc = QRAM_E_CUDA;
        G->graph = graph;
        if (!rc && !ok(cudaGraphInstantiate(&G->exec, G->graph, 0))) rc = QRAM_E_CUDA;
    }
    cudaStreamDestroy(cap);
    if (rc) { cudaGetLastError(); qram_graph_destroy(G); return rc; }
    *gout = G;
    return QRAM_OK;
}

int qram_graph_launch(qram_graph_t *G) {
    if (!G || !G->exec) return QRAM_E_ARG;
    DeviceGuard g(G->sim->device);
    if (!ok(cudaGraphLaunch(G->exec, G->sim->stream))) return QRAM_E_CUDA;
    G->sim->launches += (uint64_t)G->nk;
    return QRAM_OK;
}

void qram_graph_destroy(qram_graph_t *G) {
    if (!G) return;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
}

struct qram_batch {
    int device = 0;
    cudaStream_t stream = nullptr;           // the first simulator's stream
    std::vector<qram_sim *> sims;
    Params *d_params = nullptr;
    uint32_t *d_work = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int threads = 0, grid = 0;
    int nk = 0;                              // kernels per replay
};

int qram_batch_create(qram_sim_t *const *sims, uint32_t nsims, int mode, int threads, const uint64_t *traj0,
                      const uint32_t *ntraj, const double *const *gamma, qram_result_t *const *out,
                      qram_batch_t **bout) {
    if (!sims || !traj0 || !ntraj || !gamma || !out || !bout || nsims < 1 || nsims > (uint32_t)kMaxBatch ||
        (mode != 0 && mode != 1))
        return QRAM_E_ARG;
    *bout = nullptr;
    uint64_t total = 0;
    for (uint32_t q = 0; q < nsims; ++q) {
        const qram_sim *S = sims[q];
        if (!S || !gamma[q] || !out[q] || ntraj[q] == 0) return QRAM_E_ARG;
        if (S->device != sims[0]->device) return QRAM_E_ARG;
        if (S->eps > 0.0 || S->eps_gamma) return QRAM_E_ARG;             // damping only
        if (!(S->gamma_bound > 0.0)) return QRAM_E_STATE;                // no host read-back inside a capture
        total += ntraj[q];
    }
    if (total >= 0x7FFFFFFFull) return QRAM_E_ARG;
    if (threads == 0) threads = sims[0]->threads;
    if (!valid_threads(threads) || threads > 512) return QRAM_E_ARG;   // (no 1024-thread mixed launch)
    DeviceGuard g(sims[0]->device);
    qram_batch *B = new (std::nothrow) qram_batch();
    if (!B) return QRAM_E_OOM;
    B->device = sims[0]->device;
    B->stream = sims[0]->stream;
    B->threads = threads;
    B->sims.assign(sims, sims + nsims);
    size_t dyn = 0;
    int slots = 0x7FFFFFFF;
    int rc = QRAM_OK;
    std::vector<Params> host(nsims);
    MultiParams MP;
    std::memset(&MP, 0, sizeof(MP));
    for (uint32_t q = 0; q < nsims && !rc; ++q) {
        qram_sim *S = sims[q];
        // every problem runs in the batch's variant: scratch laid out for it
        if ((rc = qram_set_variant(S, threads))) break;
        if ((rc = ensure_scratch(S, S->gamma_bound))) break;
        dyn = std::max(dyn, S->dyn);
        slots = std::min(slots, S->slots);
        Params &P = host[q];
        P = base_params(S);
        P.traj0 = traj0[q]; P.ntraj = ntraj[q]; P.gamma = gamma[q]; P.mode = mode == 0 ? kPruned : kFull; P.out = out[q];
        MP.start[q + 1] = MP.start[q] + ntraj[q];
    }
    if (!rc) {
        const int b = kernel_blocks_per_sm_multi(threads, dyn);
        if (b < 1) rc = QRAM_E_CUDA;
        else B->grid = (int)std::min<uint64_t>((uint64_t)std::min(slots, sims[0]->sms * b), total);
    }
    cudaStream_t st = B->stream;
    if (!rc && (!ok(cudaMallocAsync((void **)&B->d_params, sizeof(Params) * nsims, st)) ||
                !ok(cudaMallocAsync((void **)&B->d_work, 256, st)))) {
        cudaGetLastError();
        rc = QRAM_E_OOM;
    }
    if (!rc && (!ok(cudaMemcpyAsync(B->d_params, host.data(), sizeof(Params) * nsims, cudaMemcpyHostToDevice, st)) ||
                !ok(cudaStreamSynchronize(st))))          // the host table goes out of scope
        rc = QRAM_E_CUDA;
    if (!rc) {
        MP.probs = B->d_params;
        MP.work = B->d_work;
        MP.nprob = nsims;
        MP.dyn_words = (uint32_t)(dyn / sizeof(uint32_t));
        cudaStream_t cap = nullptr;
        if (!ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) rc = QRAM_E_CUDA;
        else {
            if (!ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) rc = QRAM_E_CUDA;
            else {
                // launch order, longest first over all problems (the cost
                // score of launch_order, comparable across problems)
                uint32_t *perm = nullptr;
                if (total > (uint64_t)B->grid) {
                    int nmax = 0, tmax = 0;
                    for (uint32_t q = 0; q < nsims; ++q) {
                        nmax = std::max(nmax, sims[q]->n);
                        tmax = std::max(tmax, sims[q]->T);
                    }
                    if (ok(cudaMallocAsync((void **)&perm, (size_t)total * (sizeof(uint32_t) + sizeof(float)), cap))) {
                        if (!ok(launch_order_multi(MP, nmax, tmax, perm, reinterpret_cast<float *>(perm + total), cap)))
                            rc = QRAM_E_CUDA;
                        else { MP.perm = perm; B->nk += 2; }
                    } else {
                        cudaGetLastError();
                        perm = nullptr;
                    }
                }
                if (!rc && (!ok(cudaMemsetAsync(B->d_work, 0, sizeof(uint32_t), cap)) ||
                            !ok(launch_trajectories_multi(MP, B->grid, threads, dyn, cap))))
                    rc = QRAM_E_CUDA;
                else if (!rc)
                    B->nk++;
                if (perm) cudaFreeAsync(perm, cap);
                MP.perm = nullptr;
                cudaGraph_t graph = nullptr;
                if (!ok(cudaStreamEndCapture(cap, &graph))) rc = QRAM_E_CUDA;
                B->graph = graph;
                if (!rc && !ok(cudaGraphInstantiate(&B->exec, B->graph, 0))) rc = QRAM_E_CUDA;
            }
            cudaStreamDestroy(cap);
        }
    }
    if (rc) { cudaGetLastError(); qram_batch_destroy(B); return rc; }
    *bout = B;
    return QRAM_OK;
}

int qram_batch_launch(qram_batch_t *B) {
    if (!B || !B->exec) return QRAM_E_ARG;
    DeviceGuard g(B->device);
    if (!ok(cudaGraphLaunch(B->exec, B->stream))) return QRAM_E_CUDA;
    for (qram_sim *S : B->sims) S->launches += (uint64_t)B->nk;
    return QRAM_OK;
}

int qram_batch_grid(const qram_batch_t *B) { return B ? B->grid : 0; }

void qram_batch_destroy(qram_batch_t *B) {
    if (!B) return;
    {
        DeviceGuard g(B->device);
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        if (B->d_params) cudaFreeAsync(B->d_params, B->stream);
        if (B->d_work) cudaFreeAsync(B->d_work, B->stream);
        cudaStreamSynchronize(B->stream);
        cudaGetLastError();
    }
    delete B;
}

int qram_set_launch_ctas(qram_sim_t *S, uint32_t nctas) {
    if (!S) return QRAM_E_ARG;
    const int full = S->sms * S->blocks_per_sm;
    const int want = nctas == 0 ? full : (int)std::min<uint32_t>(nctas, (uint32_t)full);
    if (want != S->slots) {
        DeviceGuard g(S->device);
        if (S->scratch) { cudaFreeAsync(S->scratch, S->stream); S->scratch = nullptr; }
        S->slots = want;
    }
    return QRAM_OK;
}

int qram_set_variant(qram_sim_t *S, int threads) {
    if (!S || !valid_threads(threads)) return QRAM_E_ARG;
    if (threads == S->threads) return QRAM_OK;
    DeviceGuard g(S->device);
    const size_t dyn = dyn_smem_bytes(S->n, S->k, threads);   // (1024 threads: a larger block-sum area)
    const int b = kernel_blocks_per_sm(threads, dyn);
    if (b < 1) return QRAM_E_ARG;
    const bool capped = S->slots < S->sms * S->blocks_per_sm;
    S->threads = threads;
    S->dyn = dyn;
    S->blocks_per_sm = b;
    S->slots = capped ? std::min(S->slots, S->sms * b) : S->sms * b;
    if (S->scratch) { cudaFreeAsync(S->scratch, S->stream); S->scratch = nullptr; }
    return QRAM_OK;
}

int qram_get_variant(const qram_sim_t *S) { return S ? S->threads : 0; }

int qram_autotune(qram_sim_t *S, int mode, double gamma, uint32_t ntraj, uint64_t traj0, int *best_threads,
                  float *best_ms) {
    if (!S || !best_threads || ntraj == 0 || (mode != 0 && mode != 1) ||
        !(gamma >= 0.0 && gamma < gamma_limit(S->n, S->k)))
        return QRAM_E_ARG;
    DeviceGuard g(S->device);
    double *dg = nullptr;
    qram_result_t *dr = nullptr;
    cudaStream_t st = S->stream;
    if (!ok(cudaMallocAsync((void **)&dg, ntraj * 8ull, st)) || !ok(cudaMallocAsync((void **)&dr, ntraj * sizeof(qram_result_t), st))) {
        cudaGetLastError();
        if (dg) cudaFreeAsync(dg, st);
        return QRAM_E_OOM;
    }
    std::vector<double> hg(ntraj, gamma);
    int rc = ok(cudaMemcpyAsync(dg, hg.data(), ntraj * 8ull, cudaMemcpyHostToDevice, st)) ? QRAM_OK : QRAM_E_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (!ok(cudaEventCreate(&e0)) || !ok(cudaEventCreate(&e1)))) rc = QRAM_E_CUDA;
    const int variants[3] = {128, 256, 512};
    const int keep = S->threads;
    int best = keep;
    float bms = 3.4e38f;
    for (int v = 0; v < 3 && !rc; ++v) {
        if (qram_set_variant(S, variants[v]) != QRAM_OK) continue;
        // one untimed launch (scratch, caches), then one timed launch
        if ((rc = run_mode(S, mode, traj0, ntraj, dg, dr))) break;
        if (!ok(cudaEventRecord(e0, st))) { rc = QRAM_E_CUDA; break; }
        if ((rc = run_mode(S, mode, traj0, ntraj, dg, dr))) break;
        if (!ok(cudaEventRecord(e1, st)) || !ok(cudaEventSynchronize(e1))) { rc = QRAM_E_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < bms) { bms = ms; best = variants[v]; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(dg, st);
    cudaFreeAsync(dr, st);
    if (rc) { qram_set_variant(S, keep); return rc; }
    qram_set_variant(S, best);
    *best_threads = best;
    if (best_ms) *best_ms = bms;
    return QRAM_OK;
}

int qram_set_gamma_bound(qram_sim_t *S, double gmax) {
    if (!S || !(gmax >= 0.0 && gmax < gamma_limit(S->n, S->k))) return QRAM_E_ARG;
    S->gamma_bound = gmax;
    return QRAM_OK;
}

int qram_fidelity(qram_sim_t *S, const qram_result_t *res, uint32_t ntraj, double *mean, double *se) {
    if (!S || !res || !mean || !se) return QRAM_E_ARG;
    DeviceGuard g(S->device);
    if (!ok(launch_fidelity(res, ntraj, S->d_fid2, S->stream))) return QRAM_E_CUDA;
    S->launches++;
    double h[2];
    if (!ok(cudaMemcpyAsync(h, S->d_fid2, 16, cudaMemcpyDeviceToHost, S->stream))) return QRAM_E_CUDA;
    if (!ok(cudaStreamSynchronize(S->stream))) return QRAM_E_CUDA;
    *mean = h[0];
    *se = h[1];
    return QRAM_OK;
}

int qram_dump_state(qram_sim_t *S, int mode, uint64_t traj, double gamma, uint32_t cap, uint32_t *addr,
                    uint32_t *bus, uint64_t *hash, double *re, double *im, uint32_t *count) {
    if (!S || !count || (mode != 0 && mode != 1) || !(gamma >= 0.0 && gamma < gamma_limit(S->n, S->k)))
        return QRAM_E_ARG;
    if (cap && (!addr || !bus || !hash || !re || !im)) return QRAM_E_ARG;
    DeviceGuard g(S->device);
    int rc = ensure_scratch(S, gamma);
    if (rc) return rc;
    const uint32_t ecap = S->scr.ecap;
    const uint32_t W = ((1u << S->n) + 31u) >> 5;
    // one device block: gamma, dump buffers; the output block is sized once the
    // explicit entries are counted (each (column, tree state) group expands to
    // every bus word, and so does each closed-form branch)
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_g = take(8), o_cnt = take(8), o_scal = take(32), o_col = take(ecap * 4ull), o_bus = take(ecap * 4ull),
                 o_hash = take(ecap * 8ull), o_re = take(ecap * 8ull), o_im = take(ecap * 8ull), o_bb = take(W * 4ull),
                 o_ref = take(8), o_res = take(sizeof(qram_result_t)), o_n = take(8);
    char *b = nullptr, *ob = nullptr;
    if (!ok(cudaMalloc((void **)&b, off))) { cudaGetLastError(); return QRAM_E_OOM; }
    rc = QRAM_OK;
    do {
        if (!ok(cudaMemsetAsync(b, 0, off, S->stream))) { rc = QRAM_E_CUDA; break; }
        if (!ok(cudaMemcpyAsync(b + o_g, &gamma, 8, cudaMemcpyHostToDevice, S->stream))) { rc = QRAM_E_CUDA; break; }
        Params P = base_params(S);
        P.traj0 = traj; P.ntraj = 1; P.gamma = (const double *)(b + o_g);
        P.mode = mode == 0 ? kPruned : kFull;
        P.out = (qram_result_t *)(b + o_res);
        P.dump_mode = 1;
        P.dump_wmax = S->dump_wmax;
        P.dump.col = (uint32_t *)(b + o_col); P.dump.bus = (uint32_t *)(b + o_bus); P.dump.hash = (uint64_t *)(b + o_hash);
        P.dump.re = (double *)(b + o_re); P.dump.im = (double *)(b + o_im); P.dump.cap = ecap;
        P.dump.count = (uint32_t *)(b + o_cnt); P.dump.scal = (double *)(b + o_scal);
        P.o_badbits = (uint32_t *)(b + o_bb); P.o_ref = (int32_t *)(b + o_ref);
        if ((rc = launch(S, P, 1, gamma))) break;
        uint32_t nin = 0;
        if (!ok(cudaMemcpyAsync(&nin, b + o_cnt, 4, cudaMemcpyDeviceToHost, S->stream)) ||
            !ok(cudaStreamSynchronize(S->stream))) { rc = QRAM_E_CUDA; break; }
        if (nin > ecap) { rc = QRAM_E_CAP; break; }
        const uint64_t nw = S->enc == QRAM_QUBIT ? (uint64_t)1 << S->k : 1;
        const uint64_t ocap64 = ((uint64_t)nin + (uint64_t)S->D) * nw + 16;
        if (ocap64 > 0xFFFFFFFFull) { rc = QRAM_E_CAP; break; }
        const uint32_t ocap = (uint32_t)ocap64;
        size_t ooff = 0;
        auto otake = [&](size_t bytes) { size_t o = ooff; ooff = align_up(ooff + bytes); return o; };
        const size_t o_oa = otake(ocap * 4ull), o_ob = otake(ocap * 4ull), o_oh = otake(ocap * 8ull),
                     o_ore = otake(ocap * 8ull), o_oim = otake(ocap * 8ull);
        if (!ok(cudaMalloc((void **)&ob, ooff))) { cudaGetLastError(); rc = QRAM_E_OOM; break; }
        if (!ok(launch_dump_finalize(P, nin, (uint32_t *)(b + o_n), ocap, (uint32_t *)(ob + o_oa), (uint32_t *)(ob + o_ob),
                                     (uint64_t *)(ob + o_oh), (double *)(ob + o_ore), (double *)(ob + o_oim), S->stream))) {
            rc = QRAM_E_CUDA; break;
        }
        S->launches++;
        uint32_t nout = 0;
        if (!ok(cudaMemcpyAsync(&nout, b + o_n, 4, cudaMemcpyDeviceToHost, S->stream)) ||
            !ok(cudaStreamSynchronize(S->stream))) { rc = QRAM_E_CUDA; break; }
        *count = nout;
        const uint32_t m = std::min(nout, std::min(cap, ocap));
        if (m) {
            if (!ok(cudaMemcpyAsync(addr, ob + o_oa, m * 4ull, cudaMemcpyDeviceToHost, S->stream)) ||
                !ok(cudaMemcpyAsync(bus, ob + o_ob, m * 4ull, cudaMemcpyDeviceToHost, S->stream)) ||
                !ok(cudaMemcpyAsync(hash, ob + o_oh, m * 8ull, cudaMemcpyDeviceToHost, S->stream)) ||
                !ok(cudaMemcpyAsync(re, ob + o_ore, m * 8ull, cudaMemcpyDeviceToHost, S->stream)) ||
                !ok(cudaMemcpyAsync(im, ob + o_oim, m * 8ull, cudaMemcpyDeviceToHost, S->stream)) ||
                !ok(cudaStreamSynchronize(S->stream))) { rc = QRAM_E_CUDA; break; }
        }
        qram_result_t R;
        if (!ok(cudaMemcpy(&R, b + o_res, sizeof(R), cudaMemcpyDeviceToHost))) { rc = QRAM_E_CUDA; break; }
        if (R.status != QRAM_OK) { rc = R.status; break; }
        if (nout > cap || nout > ocap) rc = QRAM_E_CAP;
    } while (0);
    cudaFree(b);
    if (ob) cudaFree(ob);
    return rc;
}

int qram_sync(qram_sim_t *S) {
    if (!S) return QRAM_E_ARG;
    DeviceGuard g(S->device);
    if (!ok(S->stream ? cudaStreamSynchronize(S->stream) : cudaDeviceSynchronize())) return QRAM_E_CUDA;
    if (!ok(cudaGetLastError())) return QRAM_E_CUDA;
    return QRAM_OK;
}

uint64_t qram_launch_count(const qram_sim_t *S) { return S ? S->launches : 0; }

int qram_set_depolarizing(qram_sim_t *S, double eps, int eps_equals_gamma) {
    if (!S || !(eps >= 0.0 && eps < 1.0)) return QRAM_E_ARG;
    if (S->channel == QRAM_CHANNEL_HEATING && (eps > 0.0 || eps_equals_gamma)) return QRAM_E_STATE;
    S->eps = eps;
    S->eps_gamma = eps_equals_gamma ? 1 : 0;
    return QRAM_OK;
}

int qram_set_channel(qram_sim_t *S, int channel) {
    if (!S || (channel != QRAM_CHANNEL_DAMPING && channel != QRAM_CHANNEL_DEPHASING && channel != QRAM_CHANNEL_HEATING))
        return QRAM_E_ARG;
    if (channel == QRAM_CHANNEL_HEATING && (S->eps > 0.0 || S->eps_gamma)) return QRAM_E_STATE;
    S->channel = channel;
    return QRAM_OK;
}

int qram_set_dump_weight(qram_sim_t *S, int w_max) {
    if (!S || w_max < -1) return QRAM_E_ARG;
    S->dump_wmax = w_max;
    return QRAM_OK;
}

int qram_work_counters(qram_sim_t *S, uint64_t *out, int reset) {
    if (!S || !out) return QRAM_E_ARG;
    DeviceGuard g(S->device);
    char *c = reinterpret_cast<char *>(S->d_work) + 32;
    if (!ok(cudaMemcpyAsync(out, c, 64, cudaMemcpyDeviceToHost, S->stream))) return QRAM_E_CUDA;
    if (reset && !ok(cudaMemsetAsync(c, 0, 64, S->stream))) return QRAM_E_CUDA;
    if (!ok(cudaStreamSynchronize(S->stream))) return QRAM_E_CUDA;
    return QRAM_OK;
}

// Stop a running launch of this simulator from taking new trajectories: the
// work counter is raised past any trajectory count (the CTAs finish the
// trajectory in hand and exit).  Issued on `ctrl`, a stream other than the
// simulator's.  Not part of the C ABI (used by the serving loop).
int qram_internal_cancel(qram_sim_t *S, void *ctrl) {
    static const uint32_t big = 0x7FFFFFFFu;
    if (!S) return QRAM_E_ARG;
    DeviceGuard g(S->device);
    if (!ok(cudaMemcpyAsync(S->d_work, &big, 4, cudaMemcpyHostToDevice, (cudaStream_t)ctrl))) return QRAM_E_CUDA;
    return QRAM_OK;
}

}  // extern "C"
