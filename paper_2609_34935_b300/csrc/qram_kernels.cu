// qram_kernels.cu -- sm_103a kernels of the pruned trajectory simulator.
//
// One CTA simulates one trajectory at a time and takes the next trajectory
// index from a global counter (persistent, work-stealing launch).  Per
// trajectory (Algorithm 1):
//   1. candidate sampling (Theorem 3 step 1): geometric gaps between
//      candidates over the (slice, site) pairs, one Philox4x32-10 word per
//      candidate (plus one per block of 2048 pairs); each warp takes a
//      contiguous run of blocks, so concatenating the per-warp segments
//      yields the candidates in (slice, site) order without a sort;
//   2. marking (Algorithm 1 step 1): every candidate marks bad(v), Eq. (7)
//      for qutrits and Eq. (9) for qubits, into a shared-memory bitmap;
//   3. explicit set: bad branches + the first good branch (pruned) or every
//      branch (full); the qubit encoding splits each into 2^k components
//      at creation (the first Hadamard wall only signs them, Lemma 1);
//   4. evolution in epochs that end at slices with candidates.  A component
//      is the path word of its address (2 bits per tree layer: router/data
//      slot on the address path) plus a short list of off-path excitations;
//      gates on the path word are a few bit operations, anything else takes
//      a generic slow path.  K0 is applied lazily as an integer exponent.
//   5. at a slice with candidates: mask weights (Eq. (21)), including the
//      closed-form weight of the predicted good branches before the first
//      jump; one auxiliary draw picks J in the canonical order (empty mask
//      first, then sorted (site, level) lists lexicographically, a proper
//      prefix first) by a deterministic block-wide descent;
//   6. final tree measurement and fidelity; the second Hadamard wall enters
//      only through the Walsh coefficient (-1)^(bus . b_out).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "qram_internal.h"

namespace qram {


// ---------------------------------------------------------------------------
// Philox4x32-10 from its published definition (Salmon et al., SC'11).
__device__ __forceinline__ void philox(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ double uniform53(uint64_t seed, uint32_t slice, uint32_t stream, uint64_t traj) {
    uint32_t c0 = 0, c1 = slice | (stream << 24), c2 = (uint32_t)traj, c3 = (uint32_t)(traj >> 32);
    philox(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t w = (uint64_t)c0 | ((uint64_t)c1 << 32);
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// tree helpers
__device__ __forceinline__ int layer_of(uint32_t v) { return 31 - __clz(v + 1); }
__device__ __forceinline__ uint32_t path_node(uint32_t i, int n, int L) {
    return ((1u << L) - 1u) + (i >> (n - L));
}
__device__ __forceinline__ uint32_t routed_bit(uint32_t i, int n, int l) { return (i >> (n - 1 - l)) & 1u; }
// lowest common ancestor of two nodes (heap order: children of v are 2v+1, 2v+2)
__device__ __forceinline__ uint32_t tree_lca(uint32_t u, uint32_t v) {
    uint32_t x = u + 1u, y = v + 1u;                 // 1-based: the path is the binary prefix
    const int dx = 31 - __clz(x), dy = 31 - __clz(y);
    if (dx > dy) x >>= dx - dy; else y >>= dy - dx;
    while (x != y) { x >>= 1; y >>= 1; }
    return x - 1u;
}
// u is an ancestor of r, r itself, or inside subtree(r)
__device__ __forceinline__ bool tree_related(uint32_t u, uint32_t r) {
    const uint32_t x = u + 1u, y = r + 1u;
    const int dx = 31 - __clz(x), dy = 31 - __clz(y);
    return dx <= dy ? (y >> (dy - dx)) == x : (x >> (dx - dy)) == y;
}
// spread bit L of x to bit 2L
__device__ __forceinline__ uint32_t spread2(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// bad(v): subtree(v) (Eq. (7)) or, for qubits, the family-divergence range
// of Eq. (9).  Returns the leaf range [lo, hi).
__device__ void bad_range(int enc, int n, uint32_t v, uint32_t &lo, uint32_t &hi) {
    if (enc == QRAM_QUBIT) {
        while (v != 0) {
            const uint32_t par = (v - 1) >> 1;
            const bool right = (v & 1u) == 0u;
            if (right || par == 0) break;
            v = par;
        }
        if (v == 0) { lo = 0; hi = 1u << n; return; }
    }
    const int l = layer_of(v);
    const uint32_t p = v - ((1u << l) - 1u);
    lo = p << (n - l);
    hi = (p + 1u) << (n - l);
}

// set (or clear) the addresses under node v in a bitmap over addresses
__device__ __forceinline__ void mark_leaves(uint32_t *bits, int n, uint32_t v, bool set) {
    const int l = layer_of(v);
    const uint32_t p = v - ((1u << l) - 1u);
    uint32_t lo = p << (n - l);
    const uint32_t hi = (p + 1u) << (n - l);
    while (lo < hi) {
        const uint32_t wd = lo >> 5, b0 = lo & 31u;
        const uint32_t nb = min(32u - b0, hi - lo);
        const uint32_t m = nb == 32u ? 0xFFFFFFFFu : (((1u << nb) - 1u) << b0);
        if (set) atomicOr(&bits[wd], m); else atomicAnd(&bits[wd], ~m);
        lo += nb;
    }
}

// dynamic shared memory (32-bit words): three exponent histograms, at least
// the 3 x max(threads, 512) doubles of a block sum
__host__ __device__ inline uint32_t dyn_words(int n, int k, int threads = 512) {
    const uint32_t H = (uint32_t)((2 * n + k) * (6 * n + 2 * k - 1) + 1);
    const uint32_t hist = 3u * ((H + 31u) & ~31u);
    const uint32_t part = 3u * 2u * (uint32_t)(threads > 512 ? threads : 512);
    return hist > part ? hist : part;
}

// ---------------------------------------------------------------------------
// block reductions (fixed order: deterministic for a given block size)
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

constexpr int kLook = 8;           // lazy slices evaluated per look-ahead

template <int NT>
struct Smem {
    static constexpr int NW = NT / 32;
    uint32_t badbits[512];         // 2^14 addresses
    uint32_t candbits[1024];       // M <= 32766 sites, candidates of the current slice
    uint32_t slice_off[kMaxT + 2];
    uint32_t pslice_off[kMaxT + 2];   // per-slice offsets of the depolarizing events
    double powlo[64], powhi[64];   // a^j, a^(64 j)
    double redA[NW], redB[NW], redC[NW];
    uint32_t scanw[NW];
    uint32_t wcount[NW];
    uint32_t segn[NW];             // entries of each warp's compact selection segment
    uint32_t syncmask[8];          // slices whose candidates can matter: [0..3] before a jump, [4..7] after
    uint32_t cl2;                  // path-word positions (2L + slot) holding a candidate in the current slice
    uint32_t J[kMaxJ];
    int nJ;
    uint32_t nexpl, ncomp, ncand;
    int refcol;
    uint32_t nbad;
    int t;
    int status;
    double sA, sB, sC;
    double *part;                  // 3 NT doubles of the dynamic area, zero between block sums
    double dn, al, qt[kMaxK];      // per-epoch data factors (qubit): norm^2, final overlap, 1/(1 + a^(2 m_t))
    double fdn[kMaxT];             // per trajectory: the norm^2 data factor dn after damping slices 1..s
    double fW, fO;                 // per-epoch scale of the weight sums and of the overlap sum
    double bw, a2n;                // binomial groups: (1 + a^(4n))^k and a^(2n)
    double hdat[2 * kMaxN + 1];    // per trajectory: (1 + a^(2m)) / 2 and 1 / (1 + a^(2m)), m <= 2n
    double rdat[2 * kMaxN + 1];
    uint32_t region;               // after a jump: root of the subtree that can hold excitations
    uint64_t gq[kGapBits];         // fault stream: 64-bit fixed-point (1 - gamma)^(2^m)
    uint32_t hitbits[512];         // lazy epochs: addresses under a candidate on an occupied position
    uint32_t wk[8];                // work of this trajectory (see Params::ctr)
    uint32_t haspf, pfnext;        // components in product form exist (pfnext: written during a pass)
    uint32_t anyent;               // a component of this pass has a non-empty mask
    uint32_t npres;                // direct level-0 search: codes present among the entries (list if <= 128)
    uint16_t plist[128];
    // look-ahead over lazy epochs: slices, their occupied candidate positions,
    // staging offsets, exposure tables, data factors, warp partials, hit sums
    int lz_k;
    int lz_s[kLook];
    uint32_t lz_pos[kLook], lz_off[kLook + 1];
    int16_t lz_etab[kLook][4][16];
    double lz_qt[kLook][kMaxK];
    double lz_wp[kLook][NW];
    double lz_hit[kLook];
    long long t_start;             // clock64 at the trajectory's start (watchdog)
    double fprod2[kMaxT];          // product-form lazy weights: prod_l (1 + a^(2 ov_l(s))) per slice s
    double fprod1;                 // prod_l (1 + a^(ov_l(T-1))): the final overlap
    int16_t etab[4][16];           // lazy epochs: address exposure by nibble of the address
    int16_t dtab[4][16];           // qutrit: data exposure by nibble of j (0, 1) and of j ^ d (2, 3)
    int32_t econst;                // qutrit: exposure of the routers (every address bit is excited)
};

// Block sums of doubles.  FP64 issue is scarce on this part (a warp-wide
// FP64 instruction holds a sub-partition's FP64 unit for tens of cycles), so
// instead of a shuffle tree in every warp each thread parks its partial in
// S.part (NT doubles per value, zero between uses) and one warp per value
// adds them up: lane l takes partials l, l + 32, ... and a shuffle tree
// finishes.  A row of 32 partials whose bits are all zero is skipped: adding
// +0.0 changes nothing, and -0.0 is added and cleared like any value since
// the area doubles as integer histograms.  That makes sparse sums cheap.  The
// warp leaves its area zero again.  The order is fixed: deterministic.
__device__ __forceinline__ double rows_sum(double *part, int rows, uint32_t lane) {
    double r = 0.0;
    for (int q = 0; q < rows; ++q) {
        const double x = part[q * 32 + lane];
        if (__any_sync(0xFFFFFFFFu, __double_as_longlong(x) != 0)) {   // bits: -0.0 is cleared too
            r += x;
            part[q * 32 + lane] = 0.0;
        }
    }
    return warp_sum(r);
}

template <int NT>
__device__ double block_sum(double x, double *red, Smem<NT> &S) {
    (void)red;
    double *part = S.part;
    __syncthreads();
    part[threadIdx.x] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double r = rows_sum(part, NT / 32, threadIdx.x);
        if (threadIdx.x == 0) S.sA = r;
    }
    __syncthreads();
    return S.sA;
}

// three sums at once (warps 0, 1, 2: one per value, on different
// sub-partitions), each scaled by its factor (applied once, by one thread)
template <int NT>
__device__ void block_sum3(double &a, double &b, double &c, Smem<NT> &S, double fa = 1.0, double fb = 1.0,
                           double fc = 1.0) {
    static_assert(NT >= 96, "three reducing warps");
    double *part = S.part;
    __syncthreads();
    part[threadIdx.x] = a;
    part[NT + threadIdx.x] = b;
    part[2 * NT + threadIdx.x] = c;
    __syncthreads();
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if (w < 3) {
        const double r = rows_sum(part + w * NT, NT / 32, lane);
        if (lane == 0) {
            if (w == 0) S.sA = r * fa;
            else if (w == 1) S.sB = r * fb;
            else S.sC = r * fc;
        }
    }
    __syncthreads();
    a = S.sA; b = S.sB; c = S.sC;
}

// exclusive scan of a count over the block; returns prefix, total in *tot
template <int NT>
__device__ uint32_t block_scan_count(uint32_t v, uint32_t *tot, Smem<NT> &S) {
    constexpr int NW = NT / 32;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    __syncthreads();
    if (lane == 31) S.scanw[w] = x;
    __syncthreads();
    uint32_t base = 0, all = 0;
    for (uint32_t i = 0; i < NW; ++i) { if (i < w) base += S.scanw[i]; all += S.scanw[i]; }
    *tot = all;
    return base + x - v;
}

// exclusive scan of a 0/1 flag over the block; returns prefix, total in *tot
template <int NT>
__device__ uint32_t block_scan_flag(bool f, uint32_t *tot, Smem<NT> &S) {
    constexpr int NW = NT / 32;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, f);
    const uint32_t pre = __popc(b & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) S.scanw[w] = __popc(b);
    __syncthreads();
    uint32_t base = 0, all = 0;
    for (uint32_t i = 0; i < NW; ++i) { if (i < w) base += S.scanw[i]; all += S.scanw[i]; }
    *tot = all;
    return base + pre;
}

// Entry of a warp's compact selection list (components with a non-empty
// mask at the slice being drawn): the mask's first element (16 bits), its
// size capped at 7 (the descent only asks "one element or more"), whether
// the component is a binomial group (bit 19, see kBinFlag), and for
// equal-magnitude inputs the exponent e (12 bits), from which the descent
// recomputes the weight w2u a^(2e) instead of the pass storing a double.
// (kPFKey in place of e: the weight is in the FP64 list, as for every
// entry of unequal magnitudes.)
constexpr uint32_t kPFKey = 0xFFFu;
__device__ __forceinline__ uint32_t sel_key(uint32_t c1, uint32_t mcnt, int e, bool bin) {
    return (c1 & 0xFFFFu) | (min(mcnt, 7u) << 16) | ((bin ? 1u : 0u) << 19) | ((uint32_t)e & 0xFFFu) << 20;
}

// Binomial groups (qubit).  After the gates of slice 4n+2k-1 every data
// qubit is back in the bus.  A branch whose 2^k wall configurations c are
// all alive, share one tree state, carry the exponents e0 + 2n |c| (every
// data qubit excited for its whole window, Eq. (4)) and the signs
// s0 + c.phi is held as one component: the tree state, e0, s0 and phi (in the
// bus-word field), marked by bit 29 of the packed w word.  Later gates and
// K_J act on the shared tree alike, so the group stays one: its weight is
// sum_w C(k, w) a^(2 (e0 + 2n w)), its overlap with the ideal output
// (-1)^s0 sum_w K_w(|phi ^ b_out|) a^(e0 + 2n w), K_w the Krawtchouk sums
// sum_{|c| = w} (-1)^(c . psi).
constexpr uint32_t kBinFlag = 1u << 29;

__device__ __forceinline__ int binom(int k, int w) {
    int r = 1;
    for (int q = 1; q <= w; ++q) r = r * (k - w + q) / q;
    return r;
}
// sum over c in {0,1}^k with |c| = w of (-1)^(|c & psi|), |psi| = m
__device__ __forceinline__ int kraw(int k, int w, int m) {
    int r = 0;
    for (int j = 0; j <= w && j <= m; ++j)
        if (w - j <= k - m) r += ((j & 1) ? -1 : 1) * binom(m, j) * binom(k - m, w - j);
    return r;
}

// ---------------------------------------------------------------------------
// component state: the hot part lives in registers; the off-path excitations
// (rare: only after a jump moved an item off its address path) in a small
// per-thread array xs[] that only the slow path and the mask queries touch.
struct CompR {
    uint32_t pw, pwR;    // path A (the branch's address path): bit 2L router, 2L+1 data slot of its
                         // node at layer L; pwR: level-R bits (qutrit)
    uint32_t pwB;        // qubit, after a misaligned router at layer ldiv sent items off path A:
                         // path B (layers > ldiv), whose nodes follow B's own routers
    int32_t ldiv;        // divergence layer of path B, -1 = single path
    int32_t e;           // number of K0 factors a collected
    uint32_t cb;         // bus word (register outside the tree)
    uint32_t sign;       // phase (-1)^sign
    uint32_t nexc;       // off-path excitations in xs[] (never together with path B)
};

struct Ctx {
    int enc, n;
    uint32_t i;          // address of the component's branch
    uint32_t PB;         // bit 2L = bit routed at layer L (path direction)
    const uint8_t *mem;
};

__device__ __forceinline__ Ctx make_ctx(int enc, int n, const uint8_t *mem, uint32_t i) {
    Ctx C;
    C.enc = enc; C.n = n; C.mem = mem; C.i = i;
    C.PB = spread2(__brev(i) >> (32 - n));      // routed bit of layer L = bit n-1-L of i
    return C;
}

// bit 2L of x -> bit L
__device__ __forceinline__ uint32_t compact2(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// The address whose path is B: i above the divergence, the other child at
// layer ldiv, then B's router values (an idle router routes left).
__device__ __forceinline__ uint32_t b_addr(const CompR &c, const Ctx &C) {
    if (c.ldiv < 0) return 0;
    const int sh = C.n - 1 - c.ldiv;
    const uint32_t low = (1u << sh) - 1u;
    const uint32_t rev = __brev(compact2(c.pwB)) >> (32 - C.n);
    return ((C.i ^ (1u << sh)) & ~low) | (rev & low);
}

__device__ __forceinline__ bool is_ground(const CompR &c) { return c.pw == 0 && c.pwB == 0 && c.nexc == 0; }

// ---- generic slow path: sorted list of (site << 2 | level) ----------------
struct Ents {
    uint32_t v[2 * kXcap + 8];
    int n;
};

__device__ __forceinline__ int ent_get(const Ents &E, uint32_t site) {
    for (int j = 0; j < E.n; ++j) if ((E.v[j] >> 2) == site) return (int)(E.v[j] & 3u);
    return 0;
}
__device__ void ent_sort(Ents &E) {
    for (int a = 1; a < E.n; ++a) {
        uint32_t x = E.v[a]; int b = a - 1;
        while (b >= 0 && (E.v[b] >> 2) > (x >> 2)) { E.v[b + 1] = E.v[b]; --b; }
        E.v[b + 1] = x;
    }
}
__device__ bool ent_set(Ents &E, uint32_t site, int lvl) {
    for (int j = 0; j < E.n; ++j)
        if ((E.v[j] >> 2) == site) {
            if (lvl == 0) { for (int q = j; q + 1 < E.n; ++q) E.v[q] = E.v[q + 1]; --E.n; }
            else E.v[j] = (site << 2) | (uint32_t)lvl;
            return true;
        }
    if (lvl == 0) return true;
    if (E.n >= 2 * kXcap + 8) return false;
    E.v[E.n++] = (site << 2) | (uint32_t)lvl;
    ent_sort(E);
    return true;
}

// The excited sites of a component in increasing site order, as codes
// 2*site + isR, merging path A (wA), path B (wB, address iB) and the
// off-path list (xi); returns 0xFFFFFFFF at the end.
__device__ __forceinline__ uint32_t next_site(const CompR &c, const uint16_t *xs, const Ctx &C, uint32_t iB,
                                              uint32_t &wA, uint32_t &wB, uint32_t &xi) {
    uint32_t best = 0xFFFFFFFFu, code = 0xFFFFFFFFu;
    int src = -1;
    if (wA) {
        const int b = __ffs(wA) - 1;
        best = 2u * path_node(C.i, C.n, b >> 1) + (uint32_t)(b & 1);
        code = (best << 1) | ((C.enc == QRAM_QUTRIT && ((c.pwR >> b) & 1u)) ? 1u : 0u);
        src = 0;
    }
    if (wB) {
        const int b = __ffs(wB) - 1;
        const uint32_t s = 2u * path_node(iB, C.n, b >> 1) + (uint32_t)(b & 1);
        if (s < best) { best = s; code = s << 1; src = 1; }
    }
    if (xi < c.nexc) {
        const uint32_t s = xs[xi] >> 1;
        if (s < best) { best = s; code = xs[xi]; src = 2; }
    }
    if (src == 0) wA &= wA - 1;
    else if (src == 1) wB &= wB - 1;
    else if (src == 2) ++xi;
    return code;
}

__device__ void to_ents(const CompR &c, const uint16_t *xs, const Ctx &C, Ents &E) {
    E.n = 0;
    const uint32_t iB = b_addr(c, C);
    uint32_t wA = c.pw, wB = c.pwB, xi = 0;
    for (;;) {
        const uint32_t code = next_site(c, xs, C, iB, wA, wB, xi);
        if (code == 0xFFFFFFFFu) break;
        E.v[E.n++] = ((code >> 1) << 2) | ((code & 1u) ? 2u : 1u);
    }
}

__device__ bool from_ents(CompR &c, uint16_t *xs, const Ctx &C, const Ents &E) {
    c.pw = 0; c.pwR = 0; c.pwB = 0; c.ldiv = -1; c.nexc = 0;
    for (int j = 0; j < E.n; ++j) {
        const uint32_t site = E.v[j] >> 2, lvl = E.v[j] & 3u;
        const uint32_t u = site >> 1;
        const int L = layer_of(u);
        if (L < C.n && u == path_node(C.i, C.n, L)) {
            const int b = 2 * L + (int)(site & 1u);
            c.pw |= 1u << b;
            if (lvl == 2u) c.pwR |= 1u << b;
        } else {
            if (c.nexc >= (uint32_t)kXcap) return false;
            xs[c.nexc++] = (uint16_t)((site << 1) | (lvl == 2u ? 1u : 0u));
        }
    }
    return true;
}

// One slice of gates on the generic representation (App. C gate semantics).
// Takes and returns the register state by value so that callers keep it in
// registers; *okp = 0 if a capacity was exceeded.
__device__ __noinline__ CompR slow_slice(const SliceOps op, CompR c, uint16_t *xs, const Ctx C, int *okp) {
    Ents E;
    to_ents(c, xs, C, E);
    const bool qubit = C.enc == QRAM_QUBIT;
    const int n = C.n;
    *okp = 1;
    if (op.load >= 0) {
        const uint32_t b = routed_bit(C.i, n, op.load);
        const int d0 = ent_get(E, 1);
        int nd;
        if (qubit) nd = d0 ^ (int)b;
        else { const int tgt = b ? 2 : 1; nd = d0 == 0 ? tgt : (d0 == tgt ? 0 : d0); }
        if (!ent_set(E, 1, nd)) { *okp = 0; return c; }
    }
    if (op.bus >= 0) {
        const int d0 = ent_get(E, 1);
        const uint32_t b = (c.cb >> op.bus) & 1u;
        if (qubit) {
            c.cb = (c.cb & ~(1u << op.bus)) | ((uint32_t)d0 << op.bus);
            if (!ent_set(E, 1, (int)b)) { *okp = 0; return c; }
        } else if (d0 != 1) {
            c.cb = (c.cb & ~(1u << op.bus)) | ((d0 == 2 ? 1u : 0u) << op.bus);
            if (!ent_set(E, 1, b ? 2 : 0)) { *okp = 0; return c; }
        }
    }
    for (int L = 0; L < n; ++L) {
        if (!((op.iswap >> L) & 1u)) continue;
        const uint32_t lo = (1u << L) - 1u, hi = (2u << L) - 1u;
        for (int j = 0; j < E.n; ++j) {
            const uint32_t u = E.v[j] >> 3;
            if (u >= lo && u < hi) E.v[j] ^= 4u;          // site ^= 1
        }
        ent_sort(E);
    }
    for (int L = 0; L + 1 < n; ++L) {
        if (!((op.cswap >> L) & 1u)) continue;
        const uint32_t lo = (1u << L) - 1u, hi = (2u << L) - 1u;
        uint32_t nv[2 * kXcap + 8];
        for (int j = 0; j < E.n; ++j) {
            const uint32_t site = E.v[j] >> 2, u = site >> 1;
            nv[j] = E.v[j];
            if ((site & 1u) == 0u) continue;                // routers do not move
            if (u >= lo && u < hi) {
                const int r = ent_get(E, 2 * u);
                if (!qubit && r == 0) continue;
                const uint32_t child = qubit ? 2u * u + 1u + (uint32_t)r : 2u * u + (uint32_t)r;
                nv[j] = ((2u * child + 1u) << 2) | (E.v[j] & 3u);
            } else if (u >= hi && u < 2u * hi + 1u) {
                const uint32_t par = (u - 1u) >> 1;
                const int r = ent_get(E, 2 * par);
                if (!qubit && r == 0) continue;
                const uint32_t child = qubit ? 2u * par + 1u + (uint32_t)r : 2u * par + (uint32_t)r;
                if (child == u) nv[j] = ((2u * par + 1u) << 2) | (E.v[j] & 3u);
            }
        }
        for (int j = 0; j < E.n; ++j) E.v[j] = nv[j];
        ent_sort(E);
    }
    if (op.fetch >= 0) {
        const uint32_t lo = (1u << (n - 1)) - 1u, hi = (1u << n) - 1u;
        if (qubit) {
            for (int j = 0; j < E.n; ++j) {
                const uint32_t site = E.v[j] >> 2, u = site >> 1;
                if ((site & 1u) == 0u || u < lo || u >= hi) continue;
                const uint32_t cell = 2u * (u - lo) + (uint32_t)ent_get(E, 2 * u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) c.sign ^= 1u;
            }
        } else {
            uint32_t flip[2 * kXcap + 8];
            int nf = 0;
            for (int j = 0; j < E.n; ++j) {
                const uint32_t site = E.v[j] >> 2, u = site >> 1;
                if ((site & 1u) != 0u || u < lo || u >= hi) continue;
                const uint32_t cell = 2u * (u - lo) + ((E.v[j] & 3u) == 2u ? 1u : 0u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) flip[nf++] = 2u * u + 1u;
            }
            for (int f = 0; f < nf; ++f) {
                const int d = ent_get(E, flip[f]);
                if (!ent_set(E, flip[f], d == 0 ? 2 : (d == 2 ? 0 : d))) { *okp = 0; return c; }
            }
        }
    }
    if (!from_ents(c, xs, C, E)) *okp = 0;
    return c;
}

// ---- fast path on the path words -----------------------------------------
// Handles every slice in which nothing lands outside the component's paths:
// no off-path excitation; qutrit: every active controlled swap whose on-path
// data slot is occupied is aligned with the address path; qubit: the same,
// except that one misaligned router (layer ldiv) may send items to path B,
// which is kept as a second path word as long as B's routers do not change
// under items already on B.  Returns false otherwise (generic slow path).
__device__ __forceinline__ bool fast_slice(const SliceOps &op, CompR &c, const Ctx &C) {
    if (c.nexc) return false;
    const int n = C.n;
    const uint32_t CM2 = op.cswap2;
    const bool qubit = C.enc == QRAM_QUBIT;
    int ldiv = c.ldiv;
    uint32_t mis;
    if (qubit) {
        mis = (c.pw ^ C.PB) & CM2;
        const uint32_t mv = mis & (c.pw >> 1);           // data items a router would send off path A
        if (ldiv < 0) {
            if (mv) {
                if (mv & (mv - 1)) return false;         // two divergences at once
                ldiv = (__ffs(mv) - 1) >> 1;
            }
        } else {
            if (mv & ~(3u << (2 * ldiv))) return false;  // would need a third path
            // a router of B changed by this slice moves B's path below it
            const uint32_t chg = (c.pwB ^ (c.pwB >> 1)) & op.iswap2;
            if (chg && (c.pwB >> (2 * ((__ffs(chg) - 1) >> 1) + 2))) return false;
        }
    } else {
        mis = CM2 & c.pw & (c.pwR ^ C.PB);
        if (mis & (c.pw >> 1)) return false;             // a data item would leave the path
    }
    if (op.load >= 0) {
        const uint32_t b = routed_bit(C.i, n, op.load);
        if (qubit) c.pw ^= b << 1;
        else {
            const uint32_t e0 = (c.pw >> 1) & 1u, r0 = (c.pwR >> 1) & 1u;
            if (!e0) { c.pw |= 2u; c.pwR = (c.pwR & ~2u) | (b << 1); }
            else if (r0 == b) { c.pw &= ~2u; c.pwR &= ~2u; }
        }
    }
    if (op.bus >= 0) {
        const uint32_t e0 = (c.pw >> 1) & 1u, r0 = (c.pwR >> 1) & 1u;
        const uint32_t b = (c.cb >> op.bus) & 1u;
        if (qubit) {
            c.pw = (c.pw & ~2u) | (b << 1);
            c.cb = (c.cb & ~(1u << op.bus)) | (e0 << op.bus);
        } else if (!(e0 && !r0)) {                          // a slot holding L is left alone
            c.pw = (c.pw & ~2u) | (b << 1);
            c.pwR = (c.pwR & ~2u) | (b << 1);
            c.cb = (c.cb & ~(1u << op.bus)) | (e0 << op.bus);
        }
    }
    if (op.iswap2) {
        uint32_t t = (c.pw ^ (c.pw >> 1)) & op.iswap2;
        c.pw ^= t | (t << 1);
        if (qubit) {
            t = (c.pwB ^ (c.pwB >> 1)) & op.iswap2;
            c.pwB ^= t | (t << 1);
        } else {
            t = (c.pwR ^ (c.pwR >> 1)) & op.iswap2;
            c.pwR ^= t | (t << 1);
        }
    }
    if (CM2) {
        if (qubit) {
            // aligned swaps on A; on B every router is B's own direction; at the
            // divergence layer a router pointing away from A swaps with B's top
            const bool cross = ldiv >= 0 && ((mis >> (2 * ldiv)) & 1u);
            const uint32_t SMA = (CM2 & ~mis) << 1;
            const uint32_t SMB = ldiv >= 0 ? (CM2 & (0xFFFFFFFFu << (2 * ldiv + 2))) << 1 : 0u;
            uint32_t t = (c.pw ^ (c.pw >> 2)) & SMA;
            c.pw ^= t | (t << 2);
            t = (c.pwB ^ (c.pwB >> 2)) & SMB;
            c.pwB ^= t | (t << 2);
            if (cross) {
                const int bA = 2 * ldiv + 1, bB = 2 * ldiv + 3;
                const uint32_t x = ((c.pw >> bA) ^ (c.pwB >> bB)) & 1u;
                c.pw ^= x << bA;
                c.pwB ^= x << bB;
            }
        } else {
            // a qutrit router at W swaps nothing
            const uint32_t SM = (CM2 & c.pw & ~mis) << 1;
            uint32_t t = (c.pw ^ (c.pw >> 2)) & SM;
            c.pw ^= t | (t << 2);
            t = (c.pwR ^ (c.pwR >> 2)) & SM;
            c.pwR ^= t | (t << 2);
        }
    }
    if (op.fetch >= 0) {
        const int L = n - 1;
        const uint32_t re = (c.pw >> (2 * L)) & 1u, de = (c.pw >> (2 * L + 1)) & 1u;
        if (qubit) {
            if (de) {
                const uint32_t cell = ((C.i >> 1) << 1) | re;
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) c.sign ^= 1u;
            }
            if ((c.pwB >> (2 * L + 1)) & 1u) {                // the leaf of path B
                c.ldiv = ldiv;
                const uint32_t iB = b_addr(c, C);
                const uint32_t cell = ((iB >> 1) << 1) | ((c.pwB >> (2 * L)) & 1u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) c.sign ^= 1u;
            }
        } else if (re) {
            const uint32_t cell = ((C.i >> 1) << 1) | ((c.pwR >> (2 * L)) & 1u);
            if ((__ldg(C.mem + cell) >> op.fetch) & 1u) {
                const uint32_t dR = (c.pwR >> (2 * L + 1)) & 1u;
                const uint32_t bit = 1u << (2 * L + 1);
                if (!de) { c.pw |= bit; c.pwR |= bit; }
                else if (dR) { c.pw &= ~bit; c.pwR &= ~bit; }
            }
        }
    }
    c.ldiv = (ldiv >= 0 && c.pwB == 0) ? -1 : ldiv;
    return true;
}

// ---- register generic path: path A as bits, a few other sites in registers --
// The same gate semantics as slow_slice for a component whose excitations off
// its address path (path B and the off-path list together) fit in CAP
// registers (8, else 16): path A follows the fast path's bit operations, the
// other sites form an unsorted list with compile-time indices (so it stays
// in registers), and a router of path A that points away from A exchanges
// its data slot with that list.  Returns *okp = 0, leaving c and xs
// untouched, when the list would overflow.  (The memory form keeps sorted
// lists in local memory; its insertion sorts are long chains of dependent
// local accesses, several times slower, so it is left for lists above 16.)
template <int CAP>
struct HX {
    uint32_t v[CAP];     // site << 2 | level (1: excited / L, 2: R); 0 = empty
};

template <int CAP>
__device__ __forceinline__ int hx_get(const HX<CAP> &X, uint32_t site) {
    int l = 0;
#pragma unroll
    for (int q = 0; q < CAP; ++q)
        if (X.v[q] != 0u && (X.v[q] >> 2) == site) l = (int)(X.v[q] & 3u);
    return l;
}

// set the level of a site (0 removes it); false if the list is full
template <int CAP>
__device__ __forceinline__ bool hx_set(HX<CAP> &X, uint32_t site, int lvl) {
    bool done = false;
#pragma unroll
    for (int q = 0; q < CAP; ++q)
        if (!done && X.v[q] != 0u && (X.v[q] >> 2) == site) {
            X.v[q] = lvl ? ((site << 2) | (uint32_t)lvl) : 0u;
            done = true;
        }
    if (done || lvl == 0) return true;
#pragma unroll
    for (int q = 0; q < CAP; ++q)
        if (!done && X.v[q] == 0u) { X.v[q] = (site << 2) | (uint32_t)lvl; done = true; }
    return done;
}

template <int CAP>
__device__ __forceinline__ CompR hybrid_cap(const SliceOps &op, CompR c, uint16_t *xs, const Ctx &C, int *okp) {
    *okp = 0;
    const bool qubit = C.enc == QRAM_QUBIT;
    const int n = C.n;
    if (__popc(c.pwB) + (int)c.nexc > CAP) return c;
    HX<CAP> X;
#pragma unroll
    for (int q = 0; q < CAP; ++q) X.v[q] = 0u;
    {
        const uint32_t iB = b_addr(c, C);
        for (uint32_t w = c.pwB; w; w &= w - 1u) {
            const int b = __ffs(w) - 1;
            hx_set(X, 2u * path_node(iB, n, b >> 1) + (uint32_t)(b & 1), 1);
        }
        for (uint32_t q = 0; q < c.nexc; ++q) hx_set(X, xs[q] >> 1, (xs[q] & 1u) ? 2 : 1);
    }
    uint32_t pw = c.pw, pwR = c.pwR, cb = c.cb, sign = c.sign;
    // load / bus act on d_0, which is on path A (as in fast_slice)
    if (op.load >= 0) {
        const uint32_t b = routed_bit(C.i, n, op.load);
        if (qubit) pw ^= b << 1;
        else {
            const uint32_t e0 = (pw >> 1) & 1u, r0 = (pwR >> 1) & 1u;
            if (!e0) { pw |= 2u; pwR = (pwR & ~2u) | (b << 1); }
            else if (r0 == b) { pw &= ~2u; pwR &= ~2u; }
        }
    }
    if (op.bus >= 0) {
        const uint32_t e0 = (pw >> 1) & 1u, r0 = (pwR >> 1) & 1u;
        const uint32_t b = (cb >> op.bus) & 1u;
        if (qubit) {
            pw = (pw & ~2u) | (b << 1);
            cb = (cb & ~(1u << op.bus)) | (e0 << op.bus);
        } else if (!(e0 && !r0)) {
            pw = (pw & ~2u) | (b << 1);
            pwR = (pwR & ~2u) | (b << 1);
            cb = (cb & ~(1u << op.bus)) | (e0 << op.bus);
        }
    }
    if (op.iswap) {
        uint32_t t = (pw ^ (pw >> 1)) & op.iswap2;
        pw ^= t | (t << 1);
        t = (pwR ^ (pwR >> 1)) & op.iswap2;
        pwR ^= t | (t << 1);
#pragma unroll
        for (int q = 0; q < CAP; ++q)
            if (X.v[q] != 0u && ((op.iswap >> layer_of(X.v[q] >> 3)) & 1u)) X.v[q] ^= 4u;   // router <-> data
    }
    if (op.cswap) {
        // routers do not move, so each data entry moves in place, once, by
        // the routers' values
#pragma unroll
        for (int q = 0; q < CAP; ++q) {
            const uint32_t e = X.v[q], site = e >> 2, u = site >> 1;
            if (e == 0u || !(site & 1u)) continue;
            const int L = layer_of(u);
            if (((op.cswap >> L) & 1u) && L + 1 < n && u != path_node(C.i, n, L)) {
                const int r = hx_get(X, 2u * u);
                if (!qubit && r == 0) continue;
                const uint32_t child = qubit ? 2u * u + 1u + (uint32_t)r : 2u * u + (uint32_t)r;
                X.v[q] = ((2u * child + 1u) << 2) | (e & 3u);
            } else if (L >= 1 && ((op.cswap >> (L - 1)) & 1u)) {
                const uint32_t par = (u - 1u) >> 1;
                if (par == path_node(C.i, n, L - 1)) continue;           // exchange with path A below
                const int r = hx_get(X, 2u * par);
                if (!qubit && r == 0) continue;
                const uint32_t child = qubit ? 2u * par + 1u + (uint32_t)r : 2u * par + (uint32_t)r;
                if (child == u) X.v[q] = ((2u * par + 1u) << 2) | (e & 3u);
            }
        }
        for (uint32_t m = op.cswap; m; m &= m - 1u) {
            const int L = __ffs(m) - 1;
            if (L + 1 >= n) continue;
            const uint32_t uA = path_node(C.i, n, L);
            const uint32_t re = (pw >> (2 * L)) & 1u, rR = (pwR >> (2 * L)) & 1u;
            int r;                                    // router level of A's node
            if (qubit) r = (int)re;
            else { r = re ? (rR ? 2 : 1) : 0; if (r == 0) continue; }
            const uint32_t child = qubit ? 2u * uA + 1u + (uint32_t)r : 2u * uA + (uint32_t)r;
            const int bA = 2 * L + 1, bC = 2 * L + 3;
            if (child == path_node(C.i, n, L + 1)) {   // aligned: data moves along A
                uint32_t t = ((pw >> bA) ^ (pw >> bC)) & 1u;
                pw ^= (t << bA) | (t << bC);
                t = ((pwR >> bA) ^ (pwR >> bC)) & 1u;
                pwR ^= (t << bA) | (t << bC);
            } else {                                  // A's data slot <-> the other child's
                const int lo = hx_get(X, 2u * child + 1u);
                const uint32_t ea = (pw >> bA) & 1u, ra = (pwR >> bA) & 1u;
                const int la = ea ? (ra ? 2 : 1) : 0;
                if (!hx_set(X, 2u * child + 1u, la)) return c;
                pw = (pw & ~(1u << bA)) | ((lo ? 1u : 0u) << bA);
                pwR = (pwR & ~(1u << bA)) | ((lo == 2 ? 1u : 0u) << bA);
            }
        }
    }
    if (op.fetch >= 0) {
        const int L = n - 1;
        const uint32_t lo = (1u << L) - 1u;
        const uint32_t re = (pw >> (2 * L)) & 1u, de = (pw >> (2 * L + 1)) & 1u;
        if (qubit) {
            if (de) {
                const uint32_t cell = ((C.i >> 1) << 1) | re;
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) sign ^= 1u;
            }
#pragma unroll
            for (int q = 0; q < CAP; ++q) {
                const uint32_t e = X.v[q], site = e >> 2, u = site >> 1;
                if (e == 0u || !(site & 1u) || layer_of(u) != L) continue;
                const uint32_t cell = 2u * (u - lo) + (uint32_t)hx_get(X, 2u * u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) sign ^= 1u;
            }
        } else {
            if (re) {
                const uint32_t cell = ((C.i >> 1) << 1) | ((pwR >> (2 * L)) & 1u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) {
                    const uint32_t dR = (pwR >> (2 * L + 1)) & 1u;
                    const uint32_t bit = 1u << (2 * L + 1);
                    if (!de) { pw |= bit; pwR |= bit; }
                    else if (dR) { pw &= ~bit; pwR &= ~bit; }
                }
            }
            uint32_t flip[CAP];
#pragma unroll
            for (int q = 0; q < CAP; ++q) {
                const uint32_t e = X.v[q], site = e >> 2, u = site >> 1;
                flip[q] = 0u;
                if (e == 0u || (site & 1u) || layer_of(u) != L) continue;
                const uint32_t cell = 2u * (u - lo) + ((e & 3u) == 2u ? 1u : 0u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) flip[q] = 2u * u + 2u;   // data site + 1
            }
#pragma unroll
            for (int q = 0; q < CAP; ++q) {
                if (!flip[q]) continue;
                const uint32_t ds = flip[q] - 1u;
                const int d = hx_get(X, ds);
                if (!hx_set(X, ds, d == 0 ? 2 : (d == 2 ? 0 : d))) return c;
            }
        }
    }
    // sorted off-path list (insertion into xs in site order)
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < CAP; ++q) cnt += X.v[q] != 0u ? 1u : 0u;
    uint32_t prev = 0u;
    for (uint32_t k = 0; k < cnt; ++k) {
        uint32_t best = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < CAP; ++q)
            if (X.v[q] != 0u && X.v[q] > prev && X.v[q] < best) best = X.v[q];
        const uint32_t site = best >> 2;
        xs[k] = (uint16_t)((site << 1) | ((best & 3u) == 2u ? 1u : 0u));
        prev = best;
    }
    c.pw = pw; c.pwR = qubit ? 0u : pwR; c.pwB = 0u; c.ldiv = -1; c.nexc = cnt; c.cb = cb; c.sign = sign;
    *okp = 1;
    return c;
}

__device__ __noinline__ CompR hybrid_slice(const SliceOps op, CompR c, uint16_t *xs, const Ctx C, int *okp) {
    CompR h = c;
    *okp = 0;
    if (__popc(c.pwB) + (int)c.nexc <= 8) h = hybrid_cap<8>(op, c, xs, C, okp);
    if (!*okp) h = hybrid_cap<16>(op, c, xs, C, okp);            // more items, or the list grew past 8
    return *okp ? h : c;
}

// layers holding off-path items (bit L)
__device__ __forceinline__ uint32_t xs_layers(const CompR &c, const uint16_t *xs) {
    uint32_t m = 0u;
    for (uint32_t q = 0; q < c.nexc; ++q) m |= 1u << layer_of((uint32_t)xs[q] >> 2);
    return m;
}

// Does the slice act on a layer that holds off-path items (bit L of LX)?
// Its router/data swaps act within a layer, its controlled swaps between
// layers L and L + 1, the fetch on the leaf layer; load and bus act on the
// root, which is on every path.
__device__ __forceinline__ bool slice_touches(const SliceOps &op, uint32_t LX, int n) {
    return ((op.iswap | op.cswap | (op.cswap << 1)) & LX) != 0u || (op.fetch >= 0 && ((LX >> (n - 1)) & 1u));
}

// One slice of gates.  LX = xs_layers(c, xs), kept current here.  Returns
// the form that evolved it: kPathFast (path words), kPathReg (register
// generic slice), kPathMem (memory generic slice), or 0 when a capacity was
// exceeded.
enum : int { kPathFast = 1, kPathReg = 2, kPathMem = 3 };
__device__ __forceinline__ int apply_slice(const SliceOps &op, CompR &c, uint16_t *xs, const Ctx &C, uint32_t &LX) {
    if (fast_slice(op, c, C)) return kPathFast;
    if (c.nexc && !slice_touches(op, LX, C.n)) {
        // the off-path items sit this slice out: path A alone, as long as no
        // item leaves it (an off-path list never coexists with a path B)
        CompR a = c;
        a.nexc = 0;
        if (fast_slice(op, a, C) && a.ldiv < 0) {
            a.nexc = c.nexc;
            c = a;
            return kPathFast;
        }
    }
    int okv;
    const CompR h = hybrid_slice(op, c, xs, C, &okv);
    if (okv) {
        c = h;
        LX = xs_layers(c, xs);
        return kPathReg;
    }
    c = slow_slice(op, c, xs, C, &okv);
    LX = xs_layers(c, xs);
    return okv ? kPathMem : 0;
}

__device__ __forceinline__ int excited_count(const CompR &c) {
    return __popc(c.pw) + __popc(c.pwB) + (int)c.nexc;
}

// Mask J(x) = C_s n X(x) in canonical order (ascending site, then level):
// checks that its first np elements equal pref[] (ascending) and returns the
// next one.  Returns -2 on a prefix mismatch, -1 if the mask equals the
// prefix.  The order is ascending code, so J(x) starts with pref exactly when
// it holds every code of pref and no other code below pref[np - 1]; the next
// element is then the smallest code above it.  No ordered walk is needed.
// xc[0..nxc): further codes of the mask (data qubits of a component in
// product form), already known to be candidates.
__device__ __forceinline__ long long mask_query(const CompR &c, const uint16_t *xs, const Ctx &C,
                                                const uint32_t *candbits, const uint32_t *pref, int np,
                                                const uint32_t *xc = nullptr, int nxc = 0) {
    const uint32_t last = np > 0 ? pref[np - 1] : 0u;
    uint32_t next = 0xFFFFFFFFu;
    int got = 0;
    bool bad = false;
    auto take = [&](uint32_t code) {
        if (np > 0 && code <= last) {
            bool in = false;
            for (int j = 0; j < np; ++j) in |= pref[j] == code;
            if (in) ++got; else bad = true;
        } else {
            next = min(next, code);
        }
    };
    for (uint32_t w = c.pw; w; w &= w - 1u) {
        const int b = __ffs(w) - 1;
        const uint32_t site = 2u * path_node(C.i, C.n, b >> 1) + (uint32_t)(b & 1);
        if (!((candbits[site >> 5] >> (site & 31u)) & 1u)) continue;
        take((site << 1) | ((C.enc == QRAM_QUTRIT && ((c.pwR >> b) & 1u)) ? 1u : 0u));
    }
    if (c.pwB) {
        const uint32_t iB = b_addr(c, C);
        for (uint32_t w = c.pwB; w; w &= w - 1u) {
            const int b = __ffs(w) - 1;
            const uint32_t site = 2u * path_node(iB, C.n, b >> 1) + (uint32_t)(b & 1);
            if ((candbits[site >> 5] >> (site & 31u)) & 1u) take(site << 1);
        }
    }
    for (uint32_t q = 0; q < c.nexc; ++q) {
        const uint32_t site = xs[q] >> 1;
        if ((candbits[site >> 5] >> (site & 31u)) & 1u) take((uint32_t)xs[q]);
    }
    for (int q = 0; q < nxc; ++q) take(xc[q]);
    if (bad || got != np) return -2;
    return next == 0xFFFFFFFFu ? -1 : (long long)next;
}

// first element (code) of the mask J(x) = C_s n X(x) and its size; the
// code is 0xFFFF... when the mask is empty.  The canonical order (ascending
// site, then level) is ascending code, so the first element is the smallest
// code: no ordered merge of paths A, B and the off-path list is needed.
// cl2 = path-word positions (2L + slot) that hold any candidate this slice:
// an excited site at another position, on or off the paths, cannot be in J.
__device__ __forceinline__ uint32_t mask_first(const CompR &c, const uint16_t *xs, const Ctx &C,
                                               const uint32_t *candbits, uint32_t cl2, uint32_t &cnt) {
    uint32_t first = 0xFFFFFFFFu;
    cnt = 0;
    for (uint32_t w = c.pw & cl2; w; w &= w - 1u) {
        const int b = __ffs(w) - 1;
        const uint32_t site = 2u * path_node(C.i, C.n, b >> 1) + (uint32_t)(b & 1);
        if (!((candbits[site >> 5] >> (site & 31u)) & 1u)) continue;
        const uint32_t code = (site << 1) | ((C.enc == QRAM_QUTRIT && ((c.pwR >> b) & 1u)) ? 1u : 0u);
        first = min(first, code);
        ++cnt;
    }
    if (c.pwB & cl2) {
        const uint32_t iB = b_addr(c, C);
        for (uint32_t w = c.pwB & cl2; w; w &= w - 1u) {
            const int b = __ffs(w) - 1;
            const uint32_t site = 2u * path_node(iB, C.n, b >> 1) + (uint32_t)(b & 1);
            if (!((candbits[site >> 5] >> (site & 31u)) & 1u)) continue;
            first = min(first, site << 1);
            ++cnt;
        }
    }
    for (uint32_t q = 0; q < c.nexc; ++q) {
        const uint32_t site = xs[q] >> 1;
        if (!((candbits[site >> 5] >> (site & 31u)) & 1u)) continue;
        first = min(first, (uint32_t)xs[q]);
        ++cnt;
    }
    return first;
}

// where a site sits in the component: 0 = path A bit b, 1 = path B bit b,
// 2 = off-path list, -1 = not excited
__device__ __forceinline__ int locate(const CompR &c, const uint16_t *xs, const Ctx &C, uint32_t iB, uint32_t site,
                                      int &b) {
    const uint32_t u = site >> 1;
    const int L = layer_of(u);
    b = 2 * L + (int)(site & 1u);
    if (L < C.n && u == path_node(C.i, C.n, L)) return ((c.pw >> b) & 1u) ? 0 : -1;
    if (c.ldiv >= 0 && L > c.ldiv && L < C.n && u == path_node(iB, C.n, L)) return ((c.pwB >> b) & 1u) ? 1 : -1;
    for (uint32_t q = 0; q < c.nexc; ++q)
        if ((xs[q] >> 1) == site) { b = (int)q; return 2; }
    return -1;
}

// does the component hold every element of J at its level? (K_J nonzero)
__device__ __forceinline__ bool holds_all(const CompR &c, const uint16_t *xs, const Ctx &C, const uint32_t *J, int nJ) {
    const uint32_t iB = b_addr(c, C);
    for (int j = 0; j < nJ; ++j) {
        const uint32_t site = J[j] >> 1, isR = J[j] & 1u;
        int b;
        const int w = locate(c, xs, C, iB, site, b);
        if (w < 0) return false;
        if (C.enc == QRAM_QUTRIT) {
            const uint32_t lv = w == 0 ? ((c.pwR >> b) & 1u) : (xs[b] & 1u);
            if (lv != isR) return false;
        }
    }
    return true;
}

// K_J clears the sites of J.  Clearing a router of path B that has items
// below it would move B's path: the component then goes to the generic
// representation.  Takes and returns the register state by value (callers
// keep it in registers); *okp = 0 if a capacity was exceeded.
__device__ __noinline__ CompR clear_site(CompR c, uint16_t *xs, const Ctx C, uint32_t site, int *okp) {
    *okp = 1;
    const uint32_t iB = b_addr(c, C);
    int b;
    const int w = locate(c, xs, C, iB, site, b);
    if (w == 0) { c.pw &= ~(1u << b); c.pwR &= ~(1u << b); return c; }
    if (w == 1) {
        if ((b & 1) == 0 && (c.pwB >> (b + 2))) {        // B's router with items below
            Ents E;
            to_ents(c, xs, C, E);
            for (int j = 0; j < E.n; ++j)
                if ((E.v[j] >> 2) == site) { for (int q = j; q + 1 < E.n; ++q) E.v[q] = E.v[q + 1]; --E.n; break; }
            if (!from_ents(c, xs, C, E)) *okp = 0;
            return c;
        }
        c.pwB &= ~(1u << b);
        if (c.pwB == 0) c.ldiv = -1;
        return c;
    }
    if (w == 2) {
        for (uint32_t r = (uint32_t)b; r + 1 < c.nexc; ++r) xs[r] = xs[r + 1];
        --c.nexc;
    }
    return c;
}

// A depolarizing fault on one site of one component: operator t is X^a Z^b
// with (a, b) the (t+1)-th pair of {0..d-1}^2 in row order (qubit: Z, X,
// XZ; qutrit: the eight Weyl operators), X|j> = |j+1 mod d>, Z|j> = w^j|j>.
// The phase goes to sign: -1 (qubit) or w^sign, w = exp(2 pi i / 3)
// (qutrit, sign in 0..2).  Path-A sites change in registers; other sites
// through the generic representation.  By value (callers keep registers);
// *okp = 0 if a capacity was exceeded.
__device__ __noinline__ CompR pauli_site(CompR c, uint16_t *xs, const Ctx C, uint32_t site, uint32_t t, int *okp) {
    *okp = 1;
    const bool qubit = C.enc == QRAM_QUBIT;
    const int d = qubit ? 2 : 3;
    const int a = ((int)t + 1) / d, bz = ((int)t + 1) % d;
    const uint32_t iB = b_addr(c, C);
    int bpos;
    const int where = locate(c, xs, C, iB, site, bpos);
    int j = 0;                                        // current level: 0 ground, 1 L / excited, 2 R
    if (where == 0) j = (!qubit && ((c.pwR >> bpos) & 1u)) ? 2 : 1;
    else if (where == 1) j = 1;
    else if (where == 2) j = (xs[bpos] & 1u) ? 2 : 1;
    const int m = (bz * j) % d;
    if (m) c.sign = qubit ? (c.sign ^ 1u) : ((c.sign + (uint32_t)m) % 3u);
    const int nj = (j + a) % d;
    if (nj == j) return c;
    const uint32_t u = site >> 1;
    const int L = layer_of(u);
    if (L < C.n && u == path_node(C.i, C.n, L)) {
        const int b = 2 * L + (int)(site & 1u);
        c.pw = (c.pw & ~(1u << b)) | ((nj ? 1u : 0u) << b);
        c.pwR = (c.pwR & ~(1u << b)) | ((nj == 2 ? 1u : 0u) << b);
        return c;
    }
    Ents E;
    to_ents(c, xs, C, E);
    if (!ent_set(E, site, nj)) { *okp = 0; return c; }
    if (!from_ents(c, xs, C, E)) *okp = 0;
    return c;
}

// ---- heating (the outlook's diagonal heating channel) --------------------
// Jumps raise ground sites: the mask J(x) is the candidate sites that x
// holds at the ground level, each with its candidate's target level (qubit:
// the excited level; qutrit: L or R, tgt[c] = 1 or 2 for candidate c).  Codes
// as for damping, site << 1 | isR; the slice's candidates cand[c0 .. c1)
// are in site order, so the first ground candidate is the first element.
__device__ __forceinline__ uint32_t heat_code(const Ctx &C, uint32_t site, const uint32_t *tgt, uint32_t q) {
    return (site << 1) | ((C.enc == QRAM_QUTRIT && tgt[q] == 2u) ? 1u : 0u);
}

__device__ uint32_t mask_first_heat(const CompR &c, const uint16_t *xs, const Ctx &C, const uint32_t *cand,
                                    const uint32_t *tgt, uint32_t c0, uint32_t c1, uint32_t &cnt) {
    const uint32_t iB = b_addr(c, C);
    uint32_t first = 0xFFFFFFFFu;
    cnt = 0;
    for (uint32_t q = c0; q < c1; ++q) {
        const uint32_t site = cand[q] & 0xFFFFu;
        int b;
        if (locate(c, xs, C, iB, site, b) >= 0) continue;          // excited: K0 there is 1, no jump
        if (first == 0xFFFFFFFFu) first = heat_code(C, site, tgt, q);
        ++cnt;
    }
    return first;
}

// the heating mask starts with pref[0 .. np): next element, -1 if equal, -2 if not
__device__ long long mask_query_heat(const CompR &c, const uint16_t *xs, const Ctx &C, const uint32_t *cand,
                                     const uint32_t *tgt, uint32_t c0, uint32_t c1, const uint32_t *pref, int np) {
    const uint32_t iB = b_addr(c, C);
    int got = 0;
    for (uint32_t q = c0; q < c1; ++q) {
        const uint32_t site = cand[q] & 0xFFFFu;
        int b;
        if (locate(c, xs, C, iB, site, b) >= 0) continue;
        const uint32_t code = heat_code(C, site, tgt, q);
        if (got < np) {
            if (code != pref[got]) return -2;
            ++got;
            continue;
        }
        return (long long)code;
    }
    return got == np ? -1 : -2;
}

// K_J of heating: every site of J at the ground level (else the component
// is annihilated), raised to its target level.  By value; *okp = 0 if a
// capacity was exceeded.
__device__ __noinline__ CompR heat_apply(CompR c, uint16_t *xs, const Ctx C, const uint32_t *J, int nJ, bool *alive,
                                        int *okp) {
    *okp = 1;
    const uint32_t iB = b_addr(c, C);
    for (int j = 0; j < nJ; ++j) {
        int b;
        if (locate(c, xs, C, iB, J[j] >> 1, b) >= 0) { *alive = false; return c; }
    }
    *alive = true;
    for (int j = 0; j < nJ; ++j) {
        const uint32_t site = J[j] >> 1;
        const int lvl = (C.enc == QRAM_QUTRIT && (J[j] & 1u)) ? 2 : 1;
        const uint32_t u = site >> 1;
        const int L = layer_of(u);
        if (L < C.n && u == path_node(C.i, C.n, L)) {
            const int bb = 2 * L + (int)(site & 1u);
            c.pw |= 1u << bb;
            if (lvl == 2) c.pwR |= 1u << bb;
            continue;
        }
        Ents E;
        to_ents(c, xs, C, E);
        if (!ent_set(E, site, lvl) || !from_ents(c, xs, C, E)) { *okp = 0; return c; }
    }
    return c;
}

// ---- product form of the data qubits (qubit, damping) ---------------------
// From the first Hadamard wall (before the gates of slice 2n+1) until the
// last data qubit is back in the bus (slice 4n+2k-1), the 2^k wall
// configurations c of a branch differ only in which data qubits are excited.
// Every gate of those slices moves slot contents as the routers direct,
// whatever the contents are (Sec. II.A; App. C), and the routers only change
// when a data qubit would be swapped into one (or loaded into at d_0).  Until
// then the configurations share the state of every other slot (the address
// part, an ordinary component) and each data qubit t has one position, one
// exposure m_t and one phase bit ph_t: configuration c is the address part
// with data qubit t excited at its position when c_t = 1, exponent
// e + sum_t c_t m_t and sign s + sum_t c_t ph_t (Lemma 1 for the exposures;
// the wall sign (-1)^(j.c) starts ph = j).  One component (kPFFlag) then
// stands for all 2^k configurations and its weight factorises,
// a^(2e) prod_t (1 + a^(2 m_t)).  A jump on a data qubit's site keeps the
// configurations with c_t = 1: its exposure and phase join e and s, and the
// qubit (now ground) becomes part of the address part.  The address part
// holds ground at every free data qubit's position, so a configuration adds
// the excitations without collisions.  Records, one word per data qubit
// (Scratch::pfr; 0 = fixed):
//   bit 31 free | bit 23 ph | bits 16-22 m | bit 15 in the bus | bits 0-14 site, or bus slot
constexpr uint32_t kPFFlag = 1u << 30;
// Cycle budget of one trajectory (about 8 s at 2 GHz, thousands of times the
// slowest trajectory of the benchmark workloads): past it the trajectory
// ends with QRAM_E_TIMEOUT instead of holding its CTA.
constexpr long long kCycleBudget = 1ll << 34;
constexpr uint32_t kPFree = 1u << 31, kPBus = 1u << 15, kPPh = 1u << 23;

__device__ __forceinline__ uint32_t pf_m(uint32_t w) { return (w >> 16) & 0x7Fu; }

__device__ __forceinline__ void pf_load(const Scratch &scr, size_t g, uint32_t *rec) {
    const uint4 *src = reinterpret_cast<const uint4 *>(scr.pfr + g * 8);
    const uint4 a = src[0], b = src[1];
    rec[0] = a.x; rec[1] = a.y; rec[2] = a.z; rec[3] = a.w;
    rec[4] = b.x; rec[5] = b.y; rec[6] = b.z; rec[7] = b.w;
}
__device__ __forceinline__ void pf_store(const Scratch &scr, size_t g, const uint32_t *rec) {
    uint4 *dst = reinterpret_cast<uint4 *>(scr.pfr + g * 8);
    dst[0] = make_uint4(rec[0], rec[1], rec[2], rec[3]);
    dst[1] = make_uint4(rec[4], rec[5], rec[6], rec[7]);
}

// router value of node v in the address part
__device__ __forceinline__ uint32_t pf_router(const CompR &c, const uint16_t *xs, const Ctx &C, uint32_t iB,
                                              uint32_t v) {
    int b;
    return locate(c, xs, C, iB, 2u * v, b) >= 0 ? 1u : 0u;
}

// Moves the free data qubits through the gates of one slice, after the
// address part went through them (the routers that a slice's controlled
// swaps and fetch read are not changed by that slice: its gates act on
// disjoint slots).  A data qubit at a leaf during a fetch takes the phase of
// its cell.  damp: K0 of the slice follows (one more exposure in the tree).
// Returns false when a data qubit would be loaded into d_0 or swapped into a
// router (the configurations would part).
__device__ __noinline__ bool pf_move(const SliceOps op, const CompR c, const uint16_t *xs, const Ctx C,
                                     uint32_t *rec, int k, bool damp) {
    const int n = C.n;
    const uint32_t iB = b_addr(c, C);
    for (int t = 0; t < k; ++t) {
        uint32_t w = rec[t];
        if (!(w & kPFree)) continue;
        uint32_t pos = w & 0x7FFFu;
        bool bus = (w & kPBus) != 0u, moved = false;
        if (op.bus >= 0) {                                               // d_0 <-> bus slot
            if (!bus && pos == 1u) { bus = true; pos = (uint32_t)op.bus; moved = true; }
            else if (bus && pos == (uint32_t)op.bus) { bus = false; pos = 1u; moved = true; }
        }
        if (op.load >= 0 && !bus && pos == 1u) return false;
        if (!bus && !moved) {
            const uint32_t u = pos >> 1;
            const int L = layer_of(u);
            if ((op.iswap >> L) & 1u) return false;
            if ((op.cswap >> L) & 1u) {                                  // down to the routed child
                pos = 2u * (2u * u + 1u + pf_router(c, xs, C, iB, u)) + 1u;
            } else if (L > 0 && ((op.cswap >> (L - 1)) & 1u)) {          // up, if the parent routes here
                const uint32_t p = (u - 1u) >> 1;
                if (2u * p + 1u + pf_router(c, xs, C, iB, p) == u) pos = 2u * p + 1u;
            } else if (op.fetch >= 0 && L == n - 1) {
                const uint32_t cell = 2u * (u - ((1u << (n - 1)) - 1u)) + pf_router(c, xs, C, iB, u);
                if ((__ldg(C.mem + cell) >> op.fetch) & 1u) w ^= kPPh;
            }
        }
        const uint32_t m = pf_m(w) + ((damp && !bus) ? 1u : 0u);
        rec[t] = kPFree | (w & kPPh) | (m << 16) | (bus ? kPBus : 0u) | pos;
    }
    return true;
}

// K_J on a component in product form (damping), then K0 on the excited
// sites outside J: a site of J held by a free data qubit fixes that qubit
// (c_t = 1; its exposure and phase join e and s); every other site of J must
// be held by the address part (else no configuration survives: *alive =
// false) and is cleared there.  By value; *okp = 0 if a capacity was exceeded.
__device__ __noinline__ CompR pf_jump(CompR c, uint16_t *xs, const Ctx C, uint32_t *rec, int k, const uint32_t *J,
                                     int nJ, bool *alive, int *okp) {
    *okp = 1;
    *alive = true;
    uint64_t dat = 0;                  // elements of J held by data qubits
    for (int j = 0; j < nJ; ++j) {
        const uint32_t site = J[j] >> 1;
        for (int t = 0; t < k; ++t) {
            const uint32_t w = rec[t];
            if ((w & kPFree) && !(w & kPBus) && (w & 0x7FFFu) == site) {
                c.e += (int)pf_m(w);
                c.sign ^= (w & kPPh) ? 1u : 0u;
                rec[t] = 0u;
                dat |= 1ull << j;
            }
        }
    }
    const uint32_t iB = b_addr(c, C);
    for (int j = 0; j < nJ; ++j) {
        int b;
        if (!((dat >> j) & 1ull) && locate(c, xs, C, iB, J[j] >> 1, b) < 0) { *alive = false; return c; }
    }
    for (int j = 0; j < nJ; ++j) {
        if ((dat >> j) & 1ull) continue;
        int okc;
        c = clear_site(c, xs, C, J[j] >> 1, &okc);
        if (!okc) *okp = 0;
    }
    c.e += excited_count(c);
    for (int t = 0; t < k; ++t) {
        const uint32_t w = rec[t];
        if ((w & kPFree) && !(w & kPBus)) rec[t] = w + (1u << 16);
    }
    return c;
}

// Configuration cw (bit t: c_t) of a component in product form as an
// explicit component (its free data qubits only; fixed ones have c_t = 1 in
// e and s already).  False if the off-path list would overflow.
__device__ __noinline__ CompR pf_config(CompR c, uint16_t *xs, const Ctx C, const uint32_t *rec, int k, uint32_t cw,
                                       int *okp) {
    *okp = 1;
    for (int t = 0; t < k; ++t) {
        const uint32_t w = rec[t];
        if (!(w & kPFree) || !((cw >> t) & 1u)) continue;
        c.e += (int)pf_m(w);
        c.sign ^= (w & kPPh) ? 1u : 0u;
        if (w & kPBus) { c.cb |= 1u << (w & 7u); continue; }
        const uint32_t site = w & 0x7FFFu, u = site >> 1;
        const int L = layer_of(u);
        if (u == path_node(C.i, C.n, L)) { c.pw |= 1u << (2 * L + 1); continue; }
        Ents E;
        to_ents(c, xs, C, E);
        if (!ent_set(E, site, 1) || !from_ents(c, xs, C, E)) { *okp = 0; return c; }
    }
    return c;
}

// The masks of a component in product form: the address part's mask plus
// the sites of the free data qubits with c_t = 1 that hold a candidate
// (T_C, at most k).  For a subset S of T_C the configurations with c = S on
// T_C have weight base * prod_{t in S} f_t, base = a^(2e) prod over the free
// data qubits outside T_C of (1 + a^(2 m_t)), f_t = a^(2 m_t).
struct PFMasks {
    double base;
    uint32_t ntc;
    uint32_t code[kMaxK];
    double f[kMaxK];
};

__device__ __forceinline__ void pf_masks(const uint32_t *rec, int k, int e, const uint32_t *candbits,
                                         const double *powlo, const double *powhi, PFMasks &M) {
    auto ap = [&](int x) { return powlo[x & 63] * powhi[(x >> 6) & 63]; };
    const double ae = ap(e);
    M.base = ae * ae;
    M.ntc = 0;
    for (int t = 0; t < k; ++t) {
        const uint32_t w = rec[t];
        if (!(w & kPFree)) continue;
        const double am = ap((int)pf_m(w)), f = am * am;
        const uint32_t site = w & 0x7FFFu;
        if (!(w & kPBus) && ((candbits[site >> 5] >> (site & 31u)) & 1u)) {
            M.code[M.ntc] = site << 1;
            M.f[M.ntc] = f;
            ++M.ntc;
        } else {
            M.base *= 1.0 + f;
        }
    }
}

// the largest exponent of a component's configurations (product form: every free data qubit excited)
__device__ __forceinline__ int pf_etop(const uint32_t *rec, int k, int e) {
    for (int t = 0; t < k; ++t)
        if (rec[t] & kPFree) e += (int)pf_m(rec[t]);
    return e;
}

// Appends this thread's entries to its warp's selection segment: nent of
// them.  Without pm the one entry of an ordinary component or binomial
// group (first code c1, size mcnt, key exponent ke, FP64 weight w when
// wlist); with pm one per non-empty mask of a component in product form
// (subset S of T_C in increasing order, skipping the empty subset when the
// address part's mask is empty), weight wf * base * prod_{t in S} f_t in the
// FP64 list.  Entries past the segment set capfail.  Warp-uniform call.
__device__ __forceinline__ void put_entries(uint32_t nent, const PFMasks *pm, uint32_t c1, uint32_t mcnt, int ke,
                                            bool bin, double w, bool wlist, double wf, uint32_t *selk, double *selw,
                                            uint32_t selseg, uint32_t &wcur, uint32_t lane, bool &capfail) {
    const uint32_t mx = __reduce_max_sync(0xFFFFFFFFu, nent);
    for (uint32_t q = 0; q < mx; ++q) {
        const bool ne = q < nent;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ne);
        if (ne) {
            const uint32_t pos = wcur + __popc(bal & ((1u << lane) - 1u));
            if (pos >= selseg) {
                capfail = true;
            } else if (!pm) {
                selk[pos] = sel_key(c1, mcnt, ke, bin);
                if (wlist) selw[pos] = w;
            } else {
                const uint32_t sb = q + (mcnt == 0 ? 1u : 0u);
                uint32_t first = c1, cnt = mcnt;
                double wt = wf * pm->base;
                for (uint32_t i = 0; i < pm->ntc; ++i)
                    if ((sb >> i) & 1u) { first = min(first, pm->code[i]); ++cnt; wt *= pm->f[i]; }
                selk[pos] = sel_key(first, cnt, (int)kPFKey, false);
                selw[pos] = wt;
            }
        }
        wcur += __popc(bal);
    }
}

// FNV-1a over the sorted (site << 2 | level) list; 0 for the ground state
__device__ __noinline__ uint64_t config_hash(const CompR c, const uint16_t *xs, const Ctx C) {
    if (is_ground(c)) return 0;
    uint64_t h = 1469598103934665603ull;
    const uint32_t iB = b_addr(c, C);
    uint32_t wA = c.pw, wB = c.pwB, xi = 0;
    for (;;) {
        const uint32_t code = next_site(c, xs, C, iB, wA, wB, xi);
        if (code == 0xFFFFFFFFu) break;
        const uint32_t v = ((code >> 1) << 2) | ((code & 1u) ? 2u : 1u);
        for (int bb = 0; bb < 4; ++bb) { h ^= (v >> (8 * bb)) & 0xFFu; h *= 1099511628211ull; }
    }
    return h ? h : 1;
}

// a^e from the two tables a^j and a^(64 j), j < 64
template <int NT>
__device__ __forceinline__ double apow(const Smem<NT> &S, int e) {
    return S.powlo[e & 63] * S.powhi[(e >> 6) & 63];
}

// packed component (see Scratch::cs)
__device__ __forceinline__ void unpack(const uint4 v, bool qubit, CompR &c, uint32_t &col, uint32_t &addr) {
    c.pw = v.x;
    c.pwR = qubit ? 0u : v.y;
    c.pwB = qubit ? v.y : 0u;
    c.e = (int32_t)(v.z & 0xFFFu);
    c.cb = (v.z >> 12) & 0xFFu;
    c.sign = ((v.z >> 20) & 1u) | (((v.w >> 28) & 1u) << 1);
    c.nexc = (v.z >> 21) & 0x3Fu;
    c.ldiv = (int32_t)((v.z >> 27) & 0xFu) - 1;
    col = v.w & 0x3FFFu;
    addr = (v.w >> 14) & 0x3FFFu;
}

__device__ __forceinline__ uint4 pack(const CompR &c, bool qubit, uint32_t col, uint32_t addr) {
    uint4 v;
    v.x = c.pw;
    v.y = qubit ? c.pwB : c.pwR;
    v.z = ((uint32_t)c.e & 0xFFFu) | ((c.cb & 0xFFu) << 12) | ((c.sign & 1u) << 20) | ((c.nexc & 0x3Fu) << 21) |
          ((uint32_t)(c.ldiv + 1) << 27);
    v.w = col | (addr << 14) | (((c.sign >> 1) & 1u) << 28);
    return v;
}

// A component's off-path list is a 64-byte slot (kXcap entries, 16-byte
// aligned: the scratch base is 256-byte aligned), moved in 16-byte pieces;
// xs must be 16-byte aligned.  Entries past nexc are don't-cares.
static_assert(kXcap % 8 == 0, "off-path slots move in 16-byte pieces");
__device__ __forceinline__ void load_exc(const Scratch &scr, size_t g, uint32_t nexc, uint16_t *xs) {
    const uint4 *src = reinterpret_cast<const uint4 *>(scr.exc + g * kXcap);
    uint4 *dst = reinterpret_cast<uint4 *>(xs);
    for (uint32_t q = 0; q < (nexc + 7u) / 8u; ++q) dst[q] = src[q];
}

__device__ __forceinline__ void store_comp(const Scratch &scr, size_t g, const CompR &c, const uint16_t *xs,
                                           bool qubit, uint32_t col, uint32_t addr) {
    scr.cs[g] = pack(c, qubit, col, addr);
    uint4 *dst = reinterpret_cast<uint4 *>(scr.exc + g * kXcap);
    const uint4 *src = reinterpret_cast<const uint4 *>(xs);
    for (uint32_t q = 0; q < (c.nexc + 7u) / 8u; ++q) dst[q] = src[q];
}

__device__ __forceinline__ double col_w2(const Params &P, uint32_t col) {
    const double re = __ldg(P.amp_re + col), im = __ldg(P.amp_im + col);
    return re * re + im * im;
}

__device__ __forceinline__ int ov(int lo, int hi, int s) {   // |[lo,hi] n [1,s]|
    const int top = s < hi ? s : hi;
    return top >= lo ? top - lo + 1 : 0;
}

// closed-form exposure of a good branch after damping layers 1..s (Eq. (14);
// Prop. 1 for the qutrit data slots)
__device__ int good_exposure(const Params &P, uint32_t col, int s) {
    const uint32_t i = __ldg(P.addr + col);
    const int n = P.n, T = P.T;
    int E = 0;
    for (int l = 0; l < n; ++l)
        if (P.enc == QRAM_QUTRIT || routed_bit(i, n, l)) E += ov(2 * l + 1, T - 2 * l - 2, s);
    if (P.enc == QRAM_QUTRIT) {
        const uint32_t j = __ldg(P.bus + col), d = __ldg(P.mem + i);
        for (int t = 0; t < P.k; ++t) {
            const int tin = 2 * n + 2 * t + 1, tf = 3 * n + 2 * t + 1, tout = 4 * n + 2 * t + 1;
            if ((j >> t) & 1u) E += ov(tin, tf - 1, s);
            if (((j ^ d) >> t) & 1u) E += ov(tf, tout - 1, s);
        }
    }
    return E;
}

// ---- lazy branches --------------------------------------------------------
// Before the first fired jump every configuration is still on its noiseless
// orbit: K0 only scales it (Eq. (14)).  Its path word at any slice follows
// from the orbit table, its weight from the closed-form exposure; explicit
// state is only needed once a jump fires, and only for the configurations
// whose mask at that slice is non-empty (the others are annihilated).

// value of an item on the orbit of address i: address bits are excited at
// level L/R (qutrit) or when 1 (qubit); data qubit t carries the wall
// configuration cw (qubit) or the bus bit j, flipped by the fetch (qutrit)
__device__ __forceinline__ uint32_t orbit_value(const Params &P, int it, int s, uint32_t i, uint32_t cw, uint32_t j,
                                                uint32_t d, uint32_t &isR) {
    const int n = P.n;
    if (it <= n) {
        const uint32_t r = routed_bit(i, n, it - 1);
        isR = r;
        return P.enc == QRAM_QUTRIT ? 1u : r;
    }
    const int t = it - 1 - n;
    if (P.enc == QRAM_QUBIT) { isR = 0; return (cw >> t) & 1u; }
    const uint32_t v = ((((P.orbit.fetched[s] >> t) & 1u) ? (j ^ d) : j) >> t) & 1u;
    isR = v;
    return v;
}

// candidates of slice s on the orbit of address i at the positions `pos`:
// *all = every configuration has a non-empty mask; the return value (qubit)
// = data qubits whose excitation at a candidate site makes it non-empty
template <typename IsCand>
__device__ __forceinline__ uint32_t orbit_hits_by(const Params &P, IsCand is_cand, uint32_t pos, int s, uint32_t i,
                                                  uint32_t j, uint32_t d, bool &all) {
    const int n = P.n;
    uint32_t tm = 0;
    all = false;
    for (uint32_t w = pos; w; w &= w - 1u) {
        const int b = __ffs(w) - 1;
        const uint32_t site = 2u * path_node(i, n, b >> 1) + (uint32_t)(b & 1);
        if (!is_cand(site)) continue;
        const int it = P.orbit.item[s][b];
        if (P.enc == QRAM_QUBIT && it > n) { tm |= 1u << (it - 1 - n); continue; }
        uint32_t isR;
        if (orbit_value(P, it, s, i, 0u, j, d, isR)) all = true;
    }
    return tm;
}
__device__ __forceinline__ uint32_t orbit_hits(const Params &P, const uint32_t *candbits, uint32_t pos, int s,
                                               uint32_t i, uint32_t j, uint32_t d, bool &all) {
    return orbit_hits_by(P, [&](uint32_t site) { return ((candbits[site >> 5] >> (site & 31u)) & 1u) != 0u; }, pos, s, i,
                         j, d, all);
}

// the explicit state of configuration cw of the branch with address i after
// the gates of slice s (exponent left to the caller)
__device__ __forceinline__ CompR orbit_state(const Params &P, int s, uint32_t i, uint32_t cw, uint32_t j, uint32_t d) {
    CompR c;
    c.pw = 0; c.pwR = 0; c.pwB = 0; c.ldiv = -1; c.e = 0; c.nexc = 0;
    for (uint32_t w = P.orbit.occ[s]; w; w &= w - 1u) {
        const int b = __ffs(w) - 1;
        uint32_t isR;
        const uint32_t v = orbit_value(P, P.orbit.item[s][b], s, i, cw, j, d, isR);
        c.pw |= v << b;
        if (P.enc == QRAM_QUTRIT) c.pwR |= (v & isR) << b;
    }
    const uint32_t bm = P.orbit.bus[s], fm = P.orbit.fetched[s];
    if (P.enc == QRAM_QUBIT) {
        c.cb = cw & bm;
        c.sign = (__popc(j & cw) + __popc(cw & d & fm)) & 1u;          // first wall, fetch phases
    } else {
        c.cb = ((j & ~fm) | ((j ^ d) & fm)) & bm;
        c.sign = 0;
    }
    return c;
}

// qubit data exposure of wall configuration cw after damping slices 1..s
__device__ __forceinline__ int data_exposure(const Params &P, uint32_t cw, int s) {
    int E = 0;
    for (int t = 0; t < P.k; ++t)
        if ((cw >> t) & 1u) E += ov(2 * P.n + 2 * t + 1, 4 * P.n + 2 * t, s);
    return E;
}

// ---------------------------------------------------------------------------
// One fault stream of a trajectory by geometric gaps over the (slice, site)
// pairs, in blocks of kGapBlock: each warp takes a contiguous run of blocks,
// one block per lane per round, counts its events, then writes them after
// those of the lower lanes, and the warp segments are concatenated into dst
// in (slice, site) order.  Events are packed (slice << 16) | site, or, with
// operator types (ntypes > 0), (slice << 18) | (type << 15) | site, the type
// being floor(word0 * ntypes / 2^32) of counter (g, r | 5 << 24).  Returns
// the number of events (block-uniform); sets QRAM_E_CAP and returns 0 on
// overflow.
template <int NT>
__device__ uint32_t sample_stream(const Params &P, Smem<NT> &S, uint64_t thr, uint32_t stream, uint32_t ntypes,
                                  uint64_t traj, uint32_t *dst) {
    constexpr int NW = NT / 32;
    const Scratch &scr = P.scr;
    const size_t slot = blockIdx.x;
    const int T = P.T;
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint32_t tl = (uint32_t)traj, th = (uint32_t)(traj >> 32);
    __syncthreads();
    if (threadIdx.x == 0) {
        S.gq[0] = 0ull - thr;                                  // 2^64 - thr
        for (int m = 0; m + 1 < kGapBits; ++m) S.gq[m + 1] = __umul64hi(S.gq[m], S.gq[m]);
    }
    __syncthreads();
    const uint32_t M = 2u * (uint32_t)P.nodes, X = (uint32_t)(T - 1) * M;
    const uint32_t nblk = (X + kGapBlock - 1) / kGapBlock;
    const uint32_t per = (nblk + NW - 1) / NW;
    const uint32_t g0 = w * per, g1 = min(nblk, g0 + per);
    uint32_t *seg = scr.wseg + (slot * NW + w) * scr.seg_cap;
    uint32_t cnt = 0, draws = 0;
    bool overflow = false;
    for (uint32_t gb = g0; gb < g1; gb += 32) {
        const uint32_t g = gb + lane;
        uint32_t mine = 0, off = 0;
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                uint32_t x = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if (lane >= (uint32_t)o) x += y;
                }
                off = cnt + x - mine;
                cnt += __shfl_sync(0xFFFFFFFFu, x, 31);
                if (mine == 0) continue;
            }
            if (g >= g1) continue;
            uint32_t pos = g * kGapBlock;
            const uint32_t end = min(pos + kGapBlock, X);
            uint32_t o0 = 0, o1 = 0, o2 = 0, o3 = 0, k = 0;
            for (uint32_t r = 0;; ++r) {
                if ((r & 1u) == 0) {
                    o0 = g; o1 = (r >> 1) | (stream << 24); o2 = tl; o3 = th;
                    philox(o0, o1, o2, o3, k0, k1);
                }
                const uint64_t u = (r & 1u) ? ((uint64_t)o2 | ((uint64_t)o3 << 32)) : ((uint64_t)o0 | ((uint64_t)o1 << 32));
                uint64_t acc = ~0ull;
                uint32_t G = 0;
#pragma unroll
                for (int m = kGapBits - 1; m >= 0; --m) {
                    const uint64_t t = __umul64hi(acc, S.gq[m]);
                    if (t > u) { acc = t; G += 1u << m; }
                }
                if (G >= end - pos) { if (pass == 0) draws += r + 1; break; }
                pos += G;
                if (pass == 0) ++mine;
                else {
                    const uint32_t q = off + k++;
                    uint32_t v;
                    if (ntypes) {
                        uint32_t w0 = g, w1 = r | (5u << 24), w2 = tl, w3 = th;
                        philox(w0, w1, w2, w3, k0, k1);
                        const uint32_t ty = (uint32_t)(((uint64_t)w0 * ntypes) >> 32);
                        v = ((1u + pos / M) << 18) | (ty << 15) | (pos % M);
                    } else {
                        v = ((1u + pos / M) << 16) | (pos % M);
                    }
                    if (q < scr.seg_cap) seg[q] = v;
                    else overflow = true;
                }
                ++pos;
            }
        }
    }
    overflow = __any_sync(0xFFFFFFFFu, overflow);
    draws = __reduce_add_sync(0xFFFFFFFFu, draws);
    if (lane == 0) { S.wcount[w] = overflow ? 0xFFFFFFFFu : cnt; atomicAdd(&S.wk[0], draws); }
    __syncthreads();
    uint32_t off = 0, tot = 0;
    bool bad = false;
    for (uint32_t q = 0; q < NW; ++q) {
        if (S.wcount[q] == 0xFFFFFFFFu) bad = true;
        else { if (q < w) off += S.wcount[q]; tot += S.wcount[q]; }
    }
    if (bad || tot > scr.cand_cap) {
        if (threadIdx.x == 0) S.status = QRAM_E_CAP;
        tot = 0;
    } else {
        for (uint32_t c = lane; c < cnt; c += 32) dst[off + c] = seg[c];
    }
    __syncthreads();
    return tot;
}

// ---------------------------------------------------------------------------
// one trajectory
template <int NT, bool DEPOL>
__device__ void run_one(const Params &P, Smem<NT> &S, uint32_t t, uint32_t *hist) {
    constexpr int NW = NT / 32;
    const uint64_t traj = (P.traj0_dev ? *P.traj0_dev : P.traj0) + t;
    const double gamma = P.gamma[t];
    const int n = P.n, T = P.T;
    const size_t slot = blockIdx.x;
    const Scratch &scr = P.scr;
    uint32_t *cand = scr.cand + slot * scr.cand_cap;
    // rates at or above gamma_lim would underflow the unnormalised weights
    // (sampling alone does not form them)
    const bool valid = gamma >= 0.0 && gamma < 1.0 && (P.mode == kSampleOnly || gamma < P.gamma_lim) &&
                       !(P.input_error && *P.input_error);

    if (P.input_error && *P.input_error) {          // inputs failed validation: touch nothing else
        if (threadIdx.x == 0 && P.out) {
            qram_result_t R;
            memset(&R, 0, sizeof(R));
            R.ref = -1;
            R.status = QRAM_E_ARG;
            P.out[t] = R;
        }
        return;
    }
    if (threadIdx.x == 0) {
        S.t_start = clock64();
        S.status = valid ? QRAM_OK : QRAM_E_ARG; S.refcol = -1; S.nbad = 0; S.nJ = 0;
        for (int q = 0; q < 8; ++q) S.wk[q] = 0;
    }
    for (int w = threadIdx.x; w < 512; w += NT) { S.badbits[w] = 0; S.hitbits[w] = 0; }
    for (int w = threadIdx.x; w < 1024; w += NT) S.candbits[w] = 0;
    __syncthreads();

    // ---- 1. candidates ------------------------------------------------------
    const uint64_t thr = valid ? (uint64_t)__double2ull_rz(gamma * 18446744073709551616.0) : 0ull;
    uint32_t ncand = 0;
    const bool use_hist = P.nhist > t && P.hist_cand != nullptr;
    if (use_hist) {
        const uint32_t o0 = P.hist_off[t], o1 = P.hist_off[t + 1];
        ncand = o1 - o0;
        if (ncand > scr.cand_cap) { if (threadIdx.x == 0) S.status = QRAM_E_CAP; ncand = scr.cand_cap; }
        for (uint32_t c = threadIdx.x; c < ncand; c += NT) {
            // a fixed history must name slices 1..T-1 and tree sites, in (slice, site) order
            const uint32_t v = P.hist_cand[o0 + c], hs = v >> 16, hq = v & 0xFFFFu;
            if (hs == 0 || hs >= (uint32_t)T || hq >= (uint32_t)P.M || (c > 0 && P.hist_cand[o0 + c - 1] >= v))
                S.status = QRAM_E_ARG;
            cand[c] = v;
        }
    } else if (valid && thr > 0) {
        ncand = sample_stream<NT>(P, S, thr, 1u, 0u, traj, cand);
    }
    __syncthreads();
    if (S.status == QRAM_E_ARG) ncand = 0;
    if (threadIdx.x == 0) S.ncand = ncand;
    // depolarizing fault events (their own stream; every branch explicit)
    const double eps = P.eps_gamma ? gamma : P.eps;
    const bool depol = DEPOL && valid && eps > 0.0 && eps < 1.0;
    // heating: every branch explicit (its jumps raise idle sites of every branch)
    const bool heat = P.channel == QRAM_CHANNEL_HEATING;
    uint32_t *pev = scr.pev + slot * scr.cand_cap;
    uint32_t npev = 0;
    if (depol) {
        const uint64_t thr_e = (uint64_t)__double2ull_rz(eps * 18446744073709551616.0);
        if (thr_e > 0) npev = sample_stream<NT>(P, S, thr_e, 4u, P.enc == QRAM_QUBIT ? 3u : 8u, traj, pev);
    }

    // per-slice offsets (candidates are sorted by (slice, site))
    if (threadIdx.x < 8) S.syncmask[threadIdx.x] = 0;   // [4..7] are set at each fired jump
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < ncand; c += NT) {
        const uint32_t s = cand[c] >> 16, q = cand[c] & 0xFFFFu;
        const int L = layer_of(q >> 1);
        if (depol || heat || ((P.occ2[s] >> (2 * L + (int)(q & 1u))) & 1u))   // a noiseless orbit can hold it excited
            atomicOr(&S.syncmask[s >> 5], 1u << (s & 31u));
        if (heat && P.enc == QRAM_QUTRIT) {               // target level of each heating candidate (stream 6)
            uint32_t w0 = q, w1 = s | (6u << 24), w2 = (uint32_t)traj, w3 = (uint32_t)(traj >> 32);
            philox(w0, w1, w2, w3, (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
            pev[c] = (w0 & 1u) ? 2u : 1u;
        }
    }
    for (int s = threadIdx.x; s <= T; s += NT) {
        uint32_t lo = 0, hi = ncand;
        const uint32_t key = (uint32_t)s << 16;
        while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if (cand[mid] < key) lo = mid + 1; else hi = mid; }
        S.slice_off[s] = lo;
        lo = 0; hi = npev;
        const uint32_t pkey = (uint32_t)s << 18;
        while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if (pev[mid] < pkey) lo = mid + 1; else hi = mid; }
        S.pslice_off[s] = lo;
    }
    // ---- 2. marking: every fault marks bad(v), whatever its type --------------
    for (uint32_t c = threadIdx.x; c < ncand + npev; c += NT) {
        uint32_t lo, hi;
        const uint32_t site = c < ncand ? (cand[c] & 0xFFFFu) : (pev[c - ncand] & 0x7FFFu);
        bad_range(P.enc, n, site >> 1, lo, hi);
        while (lo < hi) {
            const uint32_t wd = lo >> 5, b0 = lo & 31u;
            const uint32_t nb = min(32u - b0, hi - lo);
            const uint32_t m = nb == 32u ? 0xFFFFFFFFu : (((1u << nb) - 1u) << b0);
            atomicOr(&S.badbits[wd], m);
            lo += nb;
        }
    }
    __syncthreads();

    // classification: B and the reference branch (first good input column)
    {
        uint32_t nb = 0;
        int firstgood = 0x7FFFFFFF;
        for (uint32_t b = threadIdx.x; b < (uint32_t)P.D; b += NT) {
            const uint32_t i = __ldg(P.addr + b);
            if ((S.badbits[i >> 5] >> (i & 31u)) & 1u) ++nb;
            else if ((int)b < firstgood) firstgood = (int)b;
        }
        atomicAdd(&S.nbad, nb);
        __syncthreads();
        if (threadIdx.x == 0) S.refcol = 0x7FFFFFFF;
        __syncthreads();
        atomicMin(&S.refcol, firstgood);
        __syncthreads();
        if (threadIdx.x == 0 && S.refcol == 0x7FFFFFFF) S.refcol = -1;
        __syncthreads();
    }

    if (P.dump_mode) {
        const uint32_t W = ((1u << n) + 31u) >> 5;
        for (uint32_t w = threadIdx.x; w < W; w += NT) P.o_badbits[w] = S.badbits[w];
        if (threadIdx.x == 0) P.o_ref[0] = S.refcol;
    }
    if (P.mode == kSampleOnly) {
        const uint32_t W = ((1u << n) + 31u) >> 5;
        const uint32_t cap = P.o_cap;
        for (uint32_t c = threadIdx.x; c < ncand && c < cap; c += NT) P.o_cand[(size_t)t * cap + c] = cand[c];
        for (uint32_t w = threadIdx.x; w < W; w += NT) P.o_badbits[(size_t)t * W + w] = S.badbits[w];
        if (threadIdx.x == 0) {
            P.o_ncand[t] = S.status == QRAM_E_ARG ? 0xFFFFFFFFu : (S.status == QRAM_E_CAP ? 0xFFFFFFFEu : ncand);
            P.o_bad[t] = S.nbad;
            P.o_ref[t] = S.refcol;
        }
        __syncthreads();
        return;
    }

    // pruned mode keeps every branch implicit until a jump fires (the state
    // dump takes the same form: a jump-free trajectory is emitted from the
    // closed forms of every branch, a jumped one from its explicit survivors)
    const bool lazy = P.mode == kPruned && P.orbit.ok && !depol && !heat;
    // lazy epochs in product form: qubit input over every address, equal weights
    const bool factored = lazy && P.col_of != nullptr && P.w2u != nullptr && *P.w2u > 0.0;

    // ---- 3. explicit set ----------------------------------------------------
    // damping and dephasing: a = sqrt(1 - gamma) per excited site; heating:
    // a per ground site, i.e. 1 / sqrt(1 - gamma) per excited site up to a
    // factor common to every component
    const double a = heat ? 1.0 / sqrt(1.0 - (valid ? gamma : 0.0)) : sqrt(1.0 - (valid ? gamma : 0.0));
    if (threadIdx.x < 128) {                        // a^j and a^(64 j) by binary powering
        const int j = (int)threadIdx.x & 63;
        double x = a, p = 1.0;
        if (threadIdx.x >= 64) for (int q = 0; q < 6; ++q) x *= x;   // a^64
        for (int q = 0; q < 6; ++q) {
            if ((j >> q) & 1) p *= x;
            x *= x;
        }
        if (threadIdx.x < 64) S.powlo[j] = p; else S.powhi[j] = p;
    }
    __syncthreads();
    if (threadIdx.x <= 2u * (uint32_t)n) {          // data-qubit factors of Lemma 1 by exposure m
        const double am = apow(S, (int)threadIdx.x);
        const double h = 1.0 + am * am;
        S.hdat[threadIdx.x] = 0.5 * h;
        S.rdat[threadIdx.x] = 1.0 / h;
    }
    __syncthreads();
    for (int sw = (int)threadIdx.x; P.enc == QRAM_QUBIT && sw < T; sw += NT) {
        // data factors after damping slices 1..sw (Lemma 1): each data qubit
        // t contributes (1 + a^(2 m_t)) / 2 to a branch's norm^2
        double dn = 1.0;
        for (int q = 0; q < P.k; ++q) dn *= S.hdat[ov(2 * n + 2 * q + 1, 4 * n + 2 * q, sw)];
        S.fdn[sw] = dn;
    }
    for (int sw = (int)threadIdx.x; factored && sw < T; sw += NT) {
        // sum over every address of a^(2E) after damping slices 1..s: the
        // address bits enter independently (Eq. (14))
        double p2 = 1.0, p1 = 1.0;
        for (int l = 0; l < n; ++l) {
            const double x = apow(S, ov(2 * l + 1, T - 2 * l - 2, sw));
            p2 *= 1.0 + x * x;
            p1 *= 1.0 + x;
        }
        S.fprod2[sw] = p2;
        if (sw == T - 1) S.fprod1 = p1;
    }
    uint32_t *expl = scr.expl + slot * (size_t)P.D;
    if (lazy) {
        // only the size of the explicit set is reported: B plus the reference
        if (threadIdx.x == 0) S.nexpl = S.nbad + (S.refcol >= 0 ? 1u : 0u);
    } else {
        uint32_t base = 0;
        for (uint32_t b0 = 0; b0 < (uint32_t)P.D; b0 += NT) {
            const uint32_t b = b0 + threadIdx.x;
            bool take = false;
            if (b < (uint32_t)P.D) {
                const uint32_t i = __ldg(P.addr + b);
                take = P.mode == kFull || depol || heat || ((S.badbits[i >> 5] >> (i & 31u)) & 1u) || (int)b == S.refcol;
            }
            uint32_t tot;
            const uint32_t pre = block_scan_flag(take, &tot, S);
            if (take) expl[base + pre] = b;
            base += tot;
        }
        if (threadIdx.x == 0) S.nexpl = base;
    }
    __syncthreads();
    const bool qubit = P.enc == QRAM_QUBIT;
    const int kb = qubit ? P.k : 0;
    const uint32_t ncomp0 = S.nexpl << kb;
    if (ncomp0 > scr.ecap) { if (threadIdx.x == 0) S.status = QRAM_E_CAP; }
    __syncthreads();
    const size_t cbase = slot * (size_t)scr.ecap;
    // Merged components (qubit).  Until the first Hadamard wall (slice 2n+1)
    // no data qubit is in the tree, so the 2^k wall configurations of a
    // branch have the same tree state, exponent and masks; they differ only
    // in the bus word c and the wall sign (-1)^(j.c), which matter from the
    // wall on.  Before it, one component per branch stands for all 2^k
    // (multiplicity 2^mlog in every weight); at the epoch boundary forced at
    // slice 2n they are expanded into the 2^k configurations.
    // (k = 1: two configurations per branch; the forced epoch boundaries would cost more than merging saves)
    const bool mergeable = qubit && P.k >= 2 && !heat;
    int mlog = (mergeable && !lazy) ? kb : 0;
    // components created here: one per column (merged, or qutrit), or its 2^k wall configurations
    const int clog = (qubit && mlog == 0) ? kb : 0;
    const uint32_t ncreate = S.nexpl << clog;
    if (S.status == QRAM_OK && !lazy) {
        for (uint32_t r = threadIdx.x; r < ncreate; r += NT) {
            const uint32_t col = expl[r >> clog], cw = r & ((1u << clog) - 1u);
            CompR c;
            c.pw = 0; c.pwR = 0; c.pwB = 0; c.ldiv = -1; c.e = 0; c.nexc = 0;
            const uint32_t j = __ldg(P.bus + col);
            if (qubit) { c.cb = cw; c.sign = __popc(j & cw) & 1u; }   // first wall: (-1)^(j.c) (merged: c = 0)
            else { c.cb = j; c.sign = 0; }
            store_comp(scr, cbase + r, c, nullptr, qubit, col, __ldg(P.addr + col));
        }
    }
    if (threadIdx.x == 0) S.ncomp = (S.status == QRAM_OK && !lazy) ? ncreate : 0;
    __syncthreads();

    // ---- 4. epochs ----------------------------------------------------------
    // equal-magnitude inputs: weights are w2u * a^(2e), summed as integer
    // histograms over e: all; the ground tree (final epoch) or, before it,
    // the complement of the empty mask (the rarer case: one atomic less for
    // most components); signed overlap
    const double w2u = P.w2u ? *P.w2u : 0.0;
    // (a qutrit phase w^m makes the overlap complex: those weights go through FP64)
    const bool uni = w2u > 0.0 && !(depol && P.enc == QRAM_QUTRIT);
    const int H = (2 * n + P.k) * (T - 1) + 1;
    uint32_t *hall = hist, *hemp = hist + P.hist_pad;
    int32_t *hov = (int32_t *)(hist + 2 * P.hist_pad);
    int s_prev = 0;              // slice whose damping is pending (0: none)
    bool jumped = false;
    uint32_t jumps = 0, first_jump = 0, jump_sites = 0;
    const double k2 = qubit ? ldexp(1.0, -P.k) : 1.0;   // |first-wall factor|^2
    const double inv_k2 = qubit ? ldexp(1.0, P.k) : 1.0;
    if (threadIdx.x == 0) {
        double al = 1.0;                                  // (1 + a^(2n)) / 2 per fully exposed data qubit
        if (qubit) for (int q = 0; q < P.k; ++q) al *= S.hdat[n];
        S.al = al;
        const double a2n = apow(S, 2 * n), a4n = apow(S, 4 * n);
        double bw = 1.0;
        for (int q = 0; q < P.k; ++q) bw *= 1.0 + a4n;
        S.bw = bw;
        S.a2n = a2n;
    }
    // binomial groups from slice sU on (every data qubit back in the bus)
    const int sU = 4 * n + 2 * P.k - 1;
    const bool binok = mergeable && !depol;
    const uint32_t kmask = (1u << P.k) - 1u;
    // product form of the data qubits from the first wall to sU (damping).
    // After a jump, an epoch boundary before each router swap of the unload
    // in that window lets the components whose data qubit would enter a
    // router go explicit first.  (Before a jump every component is on its
    // noiseless orbit, where no data qubit meets a router swap; and before
    // the first fetch, 3n+1, no data qubit can be off its schedule: going
    // down it moves one layer per slice whatever the routers say.)
    const bool pfok = binok && P.channel == QRAM_CHANNEL_DAMPING;
    auto pfchk = [&](int s) { return s > 3 * n + 1 && s <= sU && P.ops[s].iswap != 0u; };
    if (threadIdx.x == 0) S.haspf = 0u;
    for (;;) {
        if (mlog > 0 && s_prev >= 2 * n && pfok) {
            // each merged component becomes one in product form: every data
            // qubit free in its own bus slot, no exposure, phase bit j_t
            // (first wall)
            const uint32_t nc = S.ncomp;
            for (uint32_t r = threadIdx.x; r < nc; r += NT) {
                uint4 v = scr.cs[cbase + r];
                const uint32_t j = __ldg(P.bus + (v.w & 0x3FFFu));
                uint32_t rec[8];
                for (int t = 0; t < 8; ++t)
                    rec[t] = t < P.k ? (kPFree | (((j >> t) & 1u) ? kPPh : 0u) | kPBus | (uint32_t)t) : 0u;
                v.w |= kPFFlag;
                scr.cs[cbase + r] = v;
                pf_store(scr, cbase + r, rec);
            }
            if (threadIdx.x == 0) S.haspf = nc > 0 ? 1u : 0u;
            mlog = 0;
            __syncthreads();
        }
        if (pfok && S.haspf && (s_prev == sU || (jumped && pfchk(s_prev + 1)))) {
            // At sU each component in product form becomes a binomial group
            // (every data qubit free, in its own bus slot, exposed for its
            // whole window: the group's exponents e + 2n|c| and signs
            // s + c.ph) or its explicit configurations; before a router swap
            // of the unload, the components with a free data qubit in a data
            // slot of a swapped layer go explicit.  1: output counts and
            // offsets (in the selection list area, free here); 2: top-down
            // chunks (outputs of component r start at offset >= r).
            const bool atU = s_prev == sU;
            const uint32_t isw = atU ? 0u : P.ops[s_prev + 1].iswap;
            const uint32_t nc = S.ncomp;
            uint32_t *offs = scr.selk + slot * NW * (size_t)scr.selseg;
            auto action = [&](const uint32_t *rec) {     // 0 keep, 1 binomial group, 2 explicit
                bool group = atU, risk = false;
                for (int t = 0; t < P.k; ++t) {
                    const uint32_t w = rec[t];
                    group = group && (w & kPFree) && (w & kPBus) && pf_m(w) == 2u * n;
                    if ((w & kPFree) && !(w & kPBus) && ((isw >> layer_of((w & 0x7FFFu) >> 1)) & 1u)) risk = true;
                }
                return atU ? (group ? 1 : 2) : (risk ? 2 : 0);
            };
            auto nfree = [&](const uint32_t *rec) {
                int f = 0;
                for (int t = 0; t < P.k; ++t) f += (rec[t] & kPFree) ? 1 : 0;
                return f;
            };
            uint32_t base = 0;
            for (uint32_t r0 = 0; r0 < nc; r0 += NT) {
                const uint32_t r = r0 + threadIdx.x;
                uint32_t cnt = 0;
                if (r < nc) {
                    cnt = 1;
                    if (scr.cs[cbase + r].w & kPFFlag) {
                        uint32_t rec[8];
                        pf_load(scr, cbase + r, rec);
                        if (action(rec) == 2) cnt = 1u << nfree(rec);
                    }
                }
                uint32_t tot;
                const uint32_t pre = block_scan_count(cnt, &tot, S);
                if (r < nc) offs[r] = base + pre;
                base += tot;
            }
            bool capf = false, kept = false;
            if (!atU && base == nc) {
                kept = true;                             // every component stays as it is
            } else if (base <= scr.ecap) {
                for (int r0 = ((int)nc - 1) / NT * NT; r0 >= 0; r0 -= NT) {
                    const uint32_t r = (uint32_t)r0 + threadIdx.x;
                    const bool have = r < nc;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    alignas(16) uint16_t xs[kXcap];
                    uint32_t rec[8], o = 0;
                    int act = 0;
                    if (have) {
                        v = scr.cs[cbase + r];
                        const uint32_t nx = (v.z >> 21) & 0x3Fu;
                        if (nx) load_exc(scr, cbase + r, nx, xs);
                        if (v.w & kPFFlag) { pf_load(scr, cbase + r, rec); act = action(rec); }
                        o = offs[r];
                    }
                    __syncthreads();
                    if (have) {
                        const size_t g = cbase + o;
                        const uint32_t nx = (v.z >> 21) & 0x3Fu;
                        if (act == 0) {
                            if (o != r) {
                                scr.cs[g] = v;
                                uint4 *dst = reinterpret_cast<uint4 *>(scr.exc + g * kXcap);
                                const uint4 *src = reinterpret_cast<const uint4 *>(xs);
                                for (uint32_t q = 0; q < (nx + 7u) / 8u; ++q) dst[q] = src[q];
                                if (v.w & kPFFlag) pf_store(scr, g, rec);
                            }
                            if (v.w & kPFFlag) kept = true;
                        } else if (act == 1) {
                            uint32_t phi = 0;
                            // phi by bus slot: the group's bus word is c permuted to the slots
                            for (int t = 0; t < P.k; ++t) phi |= ((rec[t] & kPPh) ? 1u : 0u) << (rec[t] & 7u);
                            CompR c; uint32_t lab, addr;
                            unpack(v, qubit, c, lab, addr);
                            uint4 g4;
                            g4.x = v.x; g4.y = v.y;
                            g4.z = ((uint32_t)c.e & 0xFFFu) | (phi << 12) | ((c.sign & 1u) << 20) | (v.z & (0x3FFu << 21));
                            g4.w = (v.w & 0x0FFFFFFFu) | kBinFlag;
                            scr.cs[g] = g4;
                            if (o != r) {
                                uint4 *dst = reinterpret_cast<uint4 *>(scr.exc + g * kXcap);
                                const uint4 *src = reinterpret_cast<const uint4 *>(xs);
                                for (uint32_t q = 0; q < (nx + 7u) / 8u; ++q) dst[q] = src[q];
                            }
                        } else {
                            CompR c; uint32_t lab, addr;
                            unpack(v, qubit, c, lab, addr);
                            const Ctx C = make_ctx(P.enc, n, P.mem, addr);
                            uint32_t fm = 0;
                            for (int t = 0; t < P.k; ++t) fm |= ((rec[t] & kPFree) ? 1u : 0u) << t;
                            // configurations over the free data qubits, in increasing order
                            uint32_t q = 0, cw = 0;
                            do {
                                alignas(16) uint16_t xd[kXcap];
                                for (uint32_t x = 0; x < nx; ++x) xd[x] = xs[x];
                                int okc;
                                const CompR d = pf_config(c, xd, C, rec, P.k, cw, &okc);
                                if (!okc) capf = true;
                                store_comp(scr, g + q, d, xd, qubit, lab, addr);
                                ++q;
                                cw = (cw - fm) & fm;
                            } while (cw != 0u);
                        }
                    }
                    __syncthreads();
                }
            } else {
                capf = true;
            }
            const bool anyk = __syncthreads_or(kept);
            if (__syncthreads_or(capf) && threadIdx.x == 0) S.status = QRAM_E_CAP;
            if (threadIdx.x == 0) {
                if (base <= scr.ecap) S.ncomp = base;
                S.haspf = anyk ? 1u : 0u;
            }
            __syncthreads();
        }
        if (mlog > 0 && s_prev >= 2 * n) {
            // expand the merged components into the 2^k wall configurations
            // (the pending K_J of slice s_prev acts on each in the pass below).
            // Top-down chunks: chunk [r0, r0 + NT) writes [r0 2^mlog, ...),
            // where every component is already read.
            const uint32_t nc = S.ncomp, m = 1u << mlog;
            for (int r0 = ((int)nc - 1) / NT * NT; r0 >= 0; r0 -= NT) {
                const uint32_t r = (uint32_t)r0 + threadIdx.x;
                const bool have = r < nc;
                CompR c;
                alignas(16) uint16_t xs[kXcap];
                uint32_t lab = 0, addr = 0;
                if (have) {
                    unpack(scr.cs[cbase + r], qubit, c, lab, addr);
                    if (c.nexc) load_exc(scr, cbase + r, c.nexc, xs);
                }
                __syncthreads();
                if (have) {
                    const uint32_t j = __ldg(P.bus + lab);
                    for (uint32_t cw = 0; cw < m; ++cw) {
                        CompR d = c;
                        d.cb = cw;
                        d.sign = c.sign ^ (__popc(j & cw) & 1u);            // first wall: (-1)^(j.c)
                        store_comp(scr, cbase + (size_t)r * m + cw, d, xs, qubit, lab, addr);
                    }
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) S.ncomp = nc << mlog;
            mlog = 0;
            __syncthreads();
        }
        // (with the product form every explicit configuration at sU comes
        // from a component that could not be a group: nothing to merge)
        if (binok && !pfok && mlog == 0 && s_prev == sU && (!lazy || jumped)) {
            // merge each branch's 2^k wall configurations into a binomial
            // group where they qualify (see kBinFlag).  A branch's
            // configurations are consecutive components.  1: the first slot
            // of each run of one column decides, staging the group component
            // per column (the selection lists are free here) and its slot in
            // expl; 2: order-preserving compaction.
            const uint32_t nc = S.ncomp, K = 1u << P.k;
            uint4 *stg = reinterpret_cast<uint4 *>(scr.selw + slot * NW * (size_t)scr.selseg);
            for (uint32_t r = threadIdx.x; r < nc; r += NT) {
                const uint4 v = scr.cs[cbase + r];
                const uint32_t col = v.w & 0x3FFFu;
                if (r > 0 && (scr.cs[cbase + r - 1].w & 0x3FFFu) == col) continue;
                bool ok = !(v.w & kBinFlag) && r + K <= nc && (scr.cs[cbase + r + K - 1].w & 0x3FFFu) == col &&
                          (r + K == nc || (scr.cs[cbase + r + K].w & 0x3FFFu) != col);
                int e0 = -1;
                uint32_t s0 = 0, phi = 0, seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                const uint32_t nx = (v.z >> 21) & 0x3Fu;
                for (uint32_t q = 0; ok && q < K; ++q) {
                    const uint4 m = scr.cs[cbase + r + q];
                    const uint32_t cb = (m.z >> 12) & 0xFFu;
                    if (m.x != v.x || m.y != v.y || (m.z >> 21) != (v.z >> 21) || (m.w & kBinFlag) || cb > kmask ||
                        ((seen[cb >> 5] >> (cb & 31u)) & 1u)) { ok = false; break; }
                    seen[cb >> 5] |= 1u << (cb & 31u);
                    for (uint32_t x = 0; x < nx && ok; ++x)
                        if (scr.exc[(cbase + r + q) * kXcap + x] != scr.exc[(cbase + r) * kXcap + x]) ok = false;
                    if (cb == 0) { e0 = (int)(m.z & 0xFFFu); s0 = (m.z >> 20) & 1u; }
                }
                for (uint32_t q = 0; ok && q < K; ++q) {             // phi from the one-qubit configurations
                    const uint4 m = scr.cs[cbase + r + q];
                    const uint32_t cb = (m.z >> 12) & 0xFFu;
                    if (__popc(cb) == 1 && (((m.z >> 20) & 1u) ^ s0)) phi |= cb;
                }
                for (uint32_t q = 0; ok && q < K; ++q) {             // exponents e0 + 2n|c|, signs s0 + c.phi
                    const uint4 m = scr.cs[cbase + r + q];
                    const uint32_t cb = (m.z >> 12) & 0xFFu;
                    if ((int)(m.z & 0xFFFu) != e0 + 2 * n * __popc(cb) ||
                        ((m.z >> 20) & 1u) != ((s0 + __popc(cb & phi)) & 1u))
                        ok = false;
                }
                uint4 g = make_uint4(0u, 0u, 0u, 0u);
                if (ok) {
                    g.x = v.x; g.y = v.y;
                    g.z = ((uint32_t)e0 & 0xFFFu) | (phi << 12) | (s0 << 20) | (v.z & (0x3FFu << 21));
                    g.w = (v.w & 0x0FFFFFFFu) | kBinFlag;
                }
                stg[col] = g;
                expl[col] = r;
            }
            __syncthreads();
            uint32_t wr = 0;
            for (uint32_t r0 = 0; r0 < nc; r0 += NT) {
                const uint32_t r = r0 + threadIdx.x;
                bool keep = false;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                alignas(16) uint16_t xs[kXcap];
                uint32_t nx = 0;
                if (r < nc) {
                    v = scr.cs[cbase + r];
                    const uint32_t col = v.w & 0x3FFFu;
                    const uint4 g = stg[col];
                    if (g.w & kBinFlag) { keep = expl[col] == r; v = g; }
                    else keep = true;
                    nx = (v.z >> 21) & 0x3Fu;
                    if (keep && nx) load_exc(scr, cbase + r, nx, xs);
                }
                uint32_t tot;
                const uint32_t pre = block_scan_flag(keep, &tot, S);    // every read of the chunk is done
                if (keep) {
                    const size_t gdst = cbase + wr + pre;
                    scr.cs[gdst] = v;
                    uint4 *dst = reinterpret_cast<uint4 *>(scr.exc + gdst * kXcap);
                    const uint4 *src = reinterpret_cast<const uint4 *>(xs);
                    for (uint32_t q = 0; q < (nx + 7u) / 8u; ++q) dst[q] = src[q];
                }
                wr += tot;
            }
            if (threadIdx.x == 0) S.ncomp = wr;
            __syncthreads();
        }
        // next slice whose candidates can matter: before the first fired jump
        // every component is on a noiseless orbit, so a candidate on a position
        // no orbit can excite leaves J empty and needs no draw; after it, only
        // candidates in the subtree a jump damaged (and on the path to it)
        int s1 = T;
        {
            // first set bit at or after s_prev + 1 of the 128-slice mask
            const uint32_t *m = jumped ? S.syncmask + 4 : S.syncmask;
            const int s0 = s_prev + 1;
            for (int wd = s0 >> 5; wd < 4; ++wd) {
                const uint32_t bits = m[wd] & (wd == (s0 >> 5) ? (0xFFFFFFFFu << (s0 & 31)) : 0xFFFFFFFFu);
                if (bits) { s1 = min(T, 32 * wd + __ffs(bits) - 1); break; }
            }
            if (mlog > 0 && s1 > 2 * n) s1 = 2 * n;          // merged components end an epoch at 2n
            // explicit configurations end an epoch at sU, where they merge into binomial groups
            if (binok && mlog == 0 && (!lazy || jumped) && s_prev < sU && s1 > sU) s1 = sU;
            if (pfok && S.haspf && jumped)                    // before a router swap of the unload
                for (int s = s_prev + 2; s <= s1 && s <= sU; ++s)
                    if (pfchk(s)) { s1 = s - 1; break; }
            // a trajectory past its cycle budget, or an epoch that would not
            // advance, goes to its final epoch (status QRAM_E_TIMEOUT)
            if (S.status == QRAM_E_TIMEOUT || s1 <= s_prev) s1 = T;
        }
        if (factored && !jumped && s1 < T && S.status == QRAM_OK) {
            // Look-ahead over lazy epochs (product-form closed weights, before
            // the first jump).  An epoch without a jump changes no state, so the
            // next candidate slices c_0 = s1 < c_1 < ... (at most kLook) are
            // evaluated together: per slice the empty-mask weight is the closed
            // form minus the hit branches' share (as in the lazy pass below),
            // their sums take one warp partial per slice and one reduction;
            // the draws are then taken in order, and the slices before the
            // first that fires are done.  That slice is left to the regular
            // epoch.  Staging (hit bitmaps, candidate sites) uses the zero
            // histogram area and leaves it zero.
            if (threadIdx.x == 0) {
                int kk = 0, x = s1;
                while (kk < kLook && x < T) {
                    S.lz_s[kk++] = x;
                    int nx = T;
                    for (int wd = (x + 1) >> 5; wd < 4; ++wd) {
                        const uint32_t bits = S.syncmask[wd] & (wd == ((x + 1) >> 5) ? (0xFFFFFFFFu << ((x + 1) & 31)) : 0xFFFFFFFFu);
                        if (bits) { nx = min(T, 32 * wd + __ffs(bits) - 1); break; }
                    }
                    x = nx;
                }
                const uint32_t W = ((1u << n) + 31u) >> 5;
                uint32_t off = (uint32_t)kk * W;
                for (int q = 0; q < kk; ++q) {
                    S.lz_off[q] = off;
                    off += S.slice_off[S.lz_s[q] + 1] - S.slice_off[S.lz_s[q]];
                    S.lz_pos[q] = 0u;
                }
                S.lz_off[kk] = off;
                S.lz_k = (kk >= 2 && off <= 3u * (uint32_t)P.hist_pad) ? kk : 0;   // (room to stage)
            }
            __syncthreads();
            const int K = S.lz_k;
            if (K >= 2) {
                const uint32_t W = ((1u << n) + 31u) >> 5;
                for (int t = (int)threadIdx.x; t < K * 64 + K * P.k; t += NT) {
                    if (t < K * 64) {                               // exposure tables of slice j (Eq. (14))
                        const int jj = t >> 6, g = (t >> 4) & 3, v = t & 15, sw = S.lz_s[jj] - 1;
                        int e = 0;
                        for (int q = 0; q < 4; ++q) {
                            const int pb = 4 * g + q, l = n - 1 - pb;
                            if (pb < n && ((v >> q) & 1)) e += ov(2 * l + 1, T - 2 * l - 2, sw);
                        }
                        S.lz_etab[jj][g][v] = (int16_t)e;
                    } else {                                        // data factors 1 / (1 + a^(2 m_t))
                        const int jj = (t - K * 64) / P.k, q = (t - K * 64) % P.k, sw = S.lz_s[jj] - 1;
                        S.lz_qt[jj][q] = S.rdat[ov(2 * n + 2 * q + 1, 4 * n + 2 * q, sw)];
                    }
                }
                for (int jj = 0; jj < K; ++jj) {                    // hit bitmaps and candidate sites
                    const int sj = S.lz_s[jj];
                    const uint32_t c0 = S.slice_off[sj], nc = S.slice_off[sj + 1] - c0;
                    for (uint32_t c = threadIdx.x; c < nc; c += NT) {
                        const uint32_t site = cand[c0 + c] & 0xFFFFu;
                        const int b = 2 * layer_of(site >> 1) + (int)(site & 1u);
                        hist[S.lz_off[jj] + c] = site;
                        if ((P.orbit.occ[sj] >> b) & 1u) {
                            mark_leaves(hist + (size_t)jj * W, n, site >> 1, true);
                            atomicOr(&S.lz_pos[jj], 1u << b);
                        }
                    }
                }
                __syncthreads();
                for (int jj = 0; jj < K; ++jj) {
                    const int sj = S.lz_s[jj];
                    const uint32_t pos = S.lz_pos[jj], *bm = hist + (size_t)jj * W, *sites = hist + S.lz_off[jj];
                    const uint32_t ns = S.lz_off[jj + 1] - S.lz_off[jj];
                    auto in_slice = [&](uint32_t site) {
                        uint32_t a0 = 0, a1 = ns;
                        while (a0 < a1) {
                            const uint32_t m = (a0 + a1) >> 1;
                            if (sites[m] < site) a0 = m + 1; else a1 = m;
                        }
                        return a0 < ns && sites[a0] == site;
                    };
                    double acc = 0.0;
                    for (uint32_t i = threadIdx.x; pos && i < (1u << n); i += NT) {
                        if (!((bm[i >> 5] >> (i & 31u)) & 1u)) continue;
                        const uint32_t b = __ldg(P.col_of + i);
                        const int E = S.lz_etab[jj][0][i & 15u] + S.lz_etab[jj][1][(i >> 4) & 15u] +
                                      S.lz_etab[jj][2][(i >> 8) & 15u] + S.lz_etab[jj][3][(i >> 12) & 15u];
                        bool all = false;
                        const uint32_t tm = orbit_hits_by(P, in_slice, pos, sj, i, __ldg(P.bus + b), __ldg(P.mem + i), all);
                        if (!all && !tm) continue;
                        const double ae = apow(S, E);
                        double qp = 1.0;
                        for (uint32_t x = tm; x; x &= x - 1u) qp *= S.lz_qt[jj][__ffs(x) - 1];
                        acc += all ? ae * ae : ae * ae * (1.0 - qp);
                    }
                    if (__any_sync(0xFFFFFFFFu, acc != 0.0)) acc = warp_sum(acc);
                    if ((threadIdx.x & 31u) == 0) S.lz_wp[jj][threadIdx.x >> 5] = acc;
                }
                __syncthreads();
                if ((int)threadIdx.x < K) {                          // one thread per slice, fixed order
                    const int jj = (int)threadIdx.x;
                    double h = 0.0;
                    for (int q = 0; q < NW; ++q) h += S.lz_wp[jj][q];
                    S.lz_hit[jj] = h;
                }
                __syncthreads();
                int jf = K;                                         // first slice whose draw fires
                for (int jj = 0; jj < K; ++jj) {
                    const int sw = S.lz_s[jj] - 1;
                    const double fw = w2u * inv_k2 * S.fdn[sw];
                    const double wt = S.fprod2[sw] * fw, we = (S.fprod2[sw] - S.lz_hit[jj]) * fw;
                    if (!(we > uniform53(P.seed, (uint32_t)S.lz_s[jj], 2u, traj) * wt)) { jf = jj; break; }
                }
                for (uint32_t w = threadIdx.x; w < S.lz_off[K]; w += NT) hist[w] = 0u;
                if (threadIdx.x == 0 && jf > 0) S.wk[2] += (uint32_t)P.D * (uint32_t)jf;
                const int sdone = jf > 0 ? S.lz_s[jf - 1] : 0;
                __syncthreads();
                if (jf > 0) {                                       // those slices are done
                    s_prev = sdone;
                    continue;
                }
            }
        }
        const bool final_epoch = s1 >= T;
        const uint32_t mc = 1u << mlog;                    // configurations per component
        const double k2m = k2 * (double)mc;
        if (threadIdx.x == 0) {
            S.cl2 = 0;
            S.pfnext = 0u;
            S.anyent = 0u;
            // data factors after damping slices 1..sw (tabulated per trajectory)
            const int sw = final_epoch ? T - 1 : s1 - 1;
            const double dn = qubit ? S.fdn[sw] : 1.0;
            if (qubit)
                for (int q = 0; q < P.k; ++q) S.qt[q] = S.rdat[ov(2 * n + 2 * q + 1, 4 * n + 2 * q, sw)];
            S.dn = dn;
            const double al = S.al;
            // lazy epochs count branches (|c|^2 without the wall factor, data
            // factors apart); explicit epochs count components (uni: |c|^2 2^-k)
            const bool lp = lazy && !jumped;
            const double w2c = uni ? w2u * inv_k2 : 1.0;
            S.fW = lp ? w2c * dn : (uni ? w2u : 1.0);
            S.fO = lp ? w2c * al : (uni ? w2u : 1.0);
        }
        if (lazy && !jumped && threadIdx.x < 128) {
            // exposure tables of the closed form (Eq. (14); Prop. 1 for the
            // qutrit data slots) after damping slices 1..sw
            const int sw = final_epoch ? T - 1 : s1 - 1;
            const int g = (threadIdx.x >> 4) & 3, v = threadIdx.x & 15;
            int e = 0;
            if (threadIdx.x < 64) {
                if (qubit)                                           // a qubit router is excited when its bit is 1
                    for (int q = 0; q < 4; ++q) {
                        const int p = 4 * g + q, l = n - 1 - p;      // address bit p is routed at layer l
                        if (p < n && ((v >> q) & 1)) e += ov(2 * l + 1, T - 2 * l - 2, sw);
                    }
                S.etab[g][v] = (int16_t)e;
            } else if (!qubit) {
                for (int q = 0; q < 4; ++q) {
                    const int t = 4 * (g & 1) + q;
                    if (t >= P.k || !((v >> q) & 1)) continue;
                    const int tin = 2 * n + 2 * t + 1, tf = 3 * n + 2 * t + 1, tout = 4 * n + 2 * t + 1;
                    e += g < 2 ? ov(tin, tf - 1, sw) : ov(tf, tout - 1, sw);
                }
                S.dtab[g][v] = (int16_t)e;
            }
            if (threadIdx.x == 64) {
                int c = 0;
                if (!qubit) for (int l = 0; l < n; ++l) c += ov(2 * l + 1, T - 2 * l - 2, sw);
                S.econst = c;
            }
        }
        __syncthreads();
        if (!final_epoch) {
            for (uint32_t c = S.slice_off[s1] + threadIdx.x; c < S.slice_off[s1 + 1]; c += NT) {
                const uint32_t site = cand[c] & 0xFFFFu;
                const int b = 2 * layer_of(site >> 1) + (int)(site & 1u);
                atomicOr(&S.candbits[site >> 5], 1u << (site & 31u));
                atomicOr(&S.cl2, 1u << b);
                if (lazy && !jumped && ((P.orbit.occ[s1] >> b) & 1u)) mark_leaves(S.hitbits, n, site >> 1, true);
            }
        }
        __syncthreads();
        const uint32_t ncomp = S.ncomp;
        const int nJ = S.nJ;
        const bool compact = s_prev > 0 && nJ > 0;
        const bool lazy_pre = lazy && !jumped;       // every branch still on its noiseless orbit
        double wsum = 0.0, wempty = 0.0, ovl = 0.0, ovi = 0.0;
        bool capfail_lazy = false;
        if (lazy_pre) {
            // closed-form weights of every branch (Eq. (14), Lemma 1): the
            // configurations of a branch share its address exposure E and
            // differ only in their data qubits, whose factors are per-epoch
            // scalars.  Equal-magnitude inputs are counted in the integer
            // histograms over E (FP64 issue is scarce); a branch with a data
            // qubit excited at a candidate keeps only the configurations
            // where those qubits are 0 in the empty-mask weight.
            const int sw = final_epoch ? T - 1 : s1 - 1;
            const uint32_t pos = final_epoch ? 0u : (S.cl2 & P.orbit.occ[s1]);
            if (factored) {
                // Every address present with equal weights (qubit): the sum of
                // a^(2E) over all branches factorises over the address bits,
                // prod_l (1 + a^(2 ov_l)); only the branches under the slice's
                // candidates (the hit bitmap) need a look, and only to take
                // their non-empty-mask weight out of the empty-mask sum.
                if (threadIdx.x == 0) {
                    wsum = S.fprod2[sw];
                    wempty = S.fprod2[sw];                   // the final orbit is the ground tree
                    if (final_epoch) ovl = S.fprod1;         // Walsh coefficient +1 on every branch
                }
                for (uint32_t i = threadIdx.x; pos && i < (1u << n); i += NT) {
                    if ((S.hitbits[i >> 5] >> (i & 31u)) & 1u) {
                        const uint32_t b = __ldg(P.col_of + i);
                        const int E = S.etab[0][i & 15u] + S.etab[1][(i >> 4) & 15u] + S.etab[2][(i >> 8) & 15u] +
                                      S.etab[3][(i >> 12) & 15u];
                        bool all = false;
                        const uint32_t tm = orbit_hits(P, S.candbits, pos, s1, i, __ldg(P.bus + b), __ldg(P.mem + i), all);
                        if (!all && !tm) continue;
                        const double ae = apow(S, E);
                        double qp = 1.0;
                        for (uint32_t x = tm; x; x &= x - 1u) qp *= S.qt[__ffs(x) - 1];
                        wempty -= all ? ae * ae : ae * ae * (1.0 - qp);
                    }
                }
            } else
            for (uint32_t b = threadIdx.x; b < (uint32_t)P.D; b += NT) {
                const uint32_t i = __ldg(P.addr + b);
                int E = S.etab[0][i & 15u] + S.etab[1][(i >> 4) & 15u] + S.etab[2][(i >> 8) & 15u] +
                        S.etab[3][(i >> 12) & 15u];
                const bool hit = pos && ((S.hitbits[i >> 5] >> (i & 31u)) & 1u);
                uint32_t j = 0, d = 0;
                if (!qubit || hit) { j = __ldg(P.bus + b); d = __ldg(P.mem + i); }
                if (!qubit) {
                    const uint32_t x = j ^ d;
                    E += S.econst + S.dtab[0][j & 15u] + S.dtab[1][(j >> 4) & 15u] + S.dtab[2][x & 15u] +
                         S.dtab[3][(x >> 4) & 15u];
                }
                bool all = false;
                uint32_t tm = 0;
                if (hit) tm = orbit_hits(P, S.candbits, pos, s1, i, j, d, all);
                double qp = 1.0;
                for (uint32_t x = tm; x; x &= x - 1u) qp *= S.qt[__ffs(x) - 1];
                if (uni) {
                    if (E >= H) { capfail_lazy = true; continue; }
                    atomicAdd(&hall[E], 1u);
                    if (final_epoch) {                      // the orbit ends in the ground tree, Walsh coefficient +1
                        atomicAdd(&hemp[E], 1u);
                        atomicAdd(&hov[E], 1);
                    } else if (all || tm) {
                        atomicAdd(&hemp[E], 1u);            // not wholly in the empty mask
                        if (!all) {
                            const double ae = apow(S, E);
                            wempty += ae * ae * qp;
                        }
                    }
                } else {
                    const double w2 = col_w2(P, b);
                    const double ae = apow(S, E);
                    const double w = w2 * ae * ae;
                    wsum += w;
                    if (final_epoch) { wempty += w; ovl += w2 * ae; }
                    else if (!all) wempty += w * qp;
                }
            }
        }
        const uint32_t ncomp_pass = lazy_pre ? 0u : ncomp;
        uint32_t wr = 0;        // write cursor (compaction)
        bool capfail = capfail_lazy;
        // this warp's segment of the compact list of components with a non-empty mask
        const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
        uint32_t *selk = scr.selk + (slot * NW + warp) * (size_t)scr.selseg;
        double *selw = scr.selw + (slot * NW + warp) * (size_t)scr.selseg;
        uint32_t wcur = 0;
        uint32_t nsl = 0;                                  // component-slices evolved by this thread
        uint32_t n2p = 0, nreg = 0, nmem = 0, noff = 0;    // by form: two paths, register / memory generic, off-path
        for (uint32_t r0 = 0; r0 < ncomp_pass; r0 += NT) {
            const uint32_t r = r0 + threadIdx.x;
            bool alive = r < ncomp_pass;
            const uint4 cur = alive ? scr.cs[cbase + r] : make_uint4(0u, 0u, 0u, 0u);
            CompR c;
            alignas(16) uint16_t xs[kXcap];
            uint32_t lab = 0, addr = 0, c1 = 0xFFFFFFFFu, mcnt = 0;
            double w = 0.0;
            uint32_t hkey = 0xFFFFFFFFu;   // histogram key: e << 3 | ground (final) or non-empty mask << 2 | overlap sign + 1
            const bool binc = alive && (cur.w & kBinFlag);   // binomial group (kBinFlag)
            const bool pfc = alive && (cur.w & kPFFlag);     // product form (kPFFlag)
            uint32_t rec[8];
            PFMasks pm;
            uint32_t nent = 0;             // selection entries of this component
            double pwf = 0.0;              // product form: weight factor of its entries
            int binm = 0;                  // final epoch, binomial group: |phi ^ b_out|
            Ctx C;
            if (alive) {
                unpack(cur, qubit, c, lab, addr);
                if (c.nexc) load_exc(scr, cbase + r, c.nexc, xs);
                C = make_ctx(P.enc, n, P.mem, addr);
                if (pfc) pf_load(scr, cbase + r, rec);
                if (s_prev > 0 && pfc) {                    // pending K_J, then K0 (product form)
                    int okp;
                    c = pf_jump(c, xs, C, rec, P.k, S.J, nJ, &alive, &okp);
                    if (!okp) capfail = true;
                } else if (s_prev > 0) {                    // pending K_J of slice s_prev
                    // damping lowers the sites of J; dephasing keeps them
                    // excited (a projection), and K0 then acts only on the
                    // excited sites outside J
                    int keep = 0;
                    if (nJ > 0 && heat) {                   // raise the ground sites of J
                        int okh;
                        c = heat_apply(c, xs, C, S.J, nJ, &alive, &okh);
                        if (!okh) capfail = true;
                        keep = nJ;
                    } else if (nJ > 0) {
                        alive = holds_all(c, xs, C, S.J, nJ);
                        if (alive && P.channel == QRAM_CHANNEL_DAMPING)
                            for (int j = 0; j < nJ; ++j) {
                                int okc;
                                c = clear_site(c, xs, C, S.J[j] >> 1, &okc);
                                if (!okc) capfail = true;
                            }
                        else keep = nJ;
                    }
                    if (alive) c.e += excited_count(c) - keep;
                }
            }
            if (alive) {
                const int slast = final_epoch ? T - 1 : s1;
                nsl += (uint32_t)(slast - s_prev);
                uint32_t LX = xs_layers(c, xs);
                noff += c.nexc ? 1u : 0u;
                for (int s = s_prev + 1; s <= slast; ++s) {
                    const int form = apply_slice(P.ops[s], c, xs, C, LX);
                    if (!form) { capfail = true; break; }
                    if (pfc && !pf_move(P.ops[s], c, xs, C, rec, P.k, s < s1)) { capfail = true; break; }
                    n2p += (form == kPathFast && c.pwB) ? 1u : 0u;
                    nreg += form == kPathReg ? 1u : 0u;
                    nmem += form == kPathMem ? 1u : 0u;
                    if (npev) {                             // depolarizing faults of slice s
                        bool okall = true;
                        for (uint32_t e = S.pslice_off[s]; e < S.pslice_off[s + 1]; ++e) {
                            const uint32_t v = pev[e];
                            int okv;
                            c = pauli_site(c, xs, C, v & 0x7FFFu, (v >> 15) & 7u, &okv);
                            if (!okv) { okall = false; break; }
                        }
                        if (!okall) { capfail = true; break; }
                        LX = xs_layers(c, xs);
                    }
                    if (s < s1) c.e += excited_count(c);     // no candidates: K0 on every site
                }
                {
                    // the largest exponent of its configurations
                    const int etop = pfc ? pf_etop(rec, P.k, c.e) : c.e + (binc ? 2 * n * P.k : 0);
                    if (etop >= 4096 || (uni && etop >= H)) capfail = true;   // exponent bound (packed in 12 bits)
                }
                if (pfc && final_epoch) capfail = true;      // (the product form ends at slice 4n+2k-1)
                if (!final_epoch) {
                    c1 = heat ? mask_first_heat(c, xs, C, cand, pev, S.slice_off[s1], S.slice_off[s1 + 1], mcnt)
                              : mask_first(c, xs, C, S.candbits, S.cl2, mcnt);
                    nent = mcnt > 0 ? 1u : 0u;
                    if (pfc) {
                        // sum over the configurations, the empty-mask part (c = 0 on T_C)
                        pf_masks(rec, P.k, c.e, S.candbits, S.powlo, S.powhi, pm);
                        pwf = uni ? 1.0 : col_w2(P, lab) * k2;
                        double wt = pm.base;
                        for (uint32_t q = 0; q < pm.ntc; ++q) wt *= 1.0 + pm.f[q];
                        wsum += pwf * wt;
                        if (mcnt == 0) wempty += pwf * pm.base;
                        nent = (1u << pm.ntc) - (mcnt == 0 ? 1u : 0u);
                    } else if (!uni) {
                        const double ae = apow(S, c.e);
                        w = col_w2(P, lab) * k2m * ae * ae * (binc ? S.bw : 1.0);
                        wsum += w;
                        if (mcnt == 0) wempty += w;
                    } else {
                        if (c.e < H) hkey = ((uint32_t)c.e << 3) | ((mcnt != 0 ? 1u : 0u) << 2) | 1u;
                    }
                } else {
                    const double ae = apow(S, c.e);
                    int ovs = 0;
                    const bool ground = is_ground(c);                 // ground tree configuration
                    if (ground) {
                        const uint32_t col = lab;
                        if (qubit) {
                            const uint32_t bout = __ldg(P.bus + col) ^ __ldg(P.mem + C.i);
                            if (binc) { binm = __popc((c.cb ^ bout) & kmask); ovs = (c.sign & 1u) ? -1 : 1; }
                            else ovs = ((c.sign + __popc(c.cb & bout)) & 1u) ? -1 : 1;
                        } else if (c.cb == (__ldg(P.bus + col) ^ __ldg(P.mem + C.i))) {
                            ovs = 1;
                        }
                    }
                    if (!uni) {
                        w = col_w2(P, lab) * k2 * ae * ae * (binc ? S.bw : 1.0);
                        wsum += w;
                        if (ground) wempty += w;
                        if (ovs) {
                            double base = col_w2(P, lab) * k2 * ae;
                            if (binc)                                 // prod over the data qubits of 1 +- a^(2n)
                                for (int q = 0; q < P.k; ++q) base *= q < binm ? 1.0 - S.a2n : 1.0 + S.a2n;
                            if (!qubit && c.sign) {                   // w^sign, w = exp(2 pi i / 3)
                                ovl -= 0.5 * base;
                                ovi += (c.sign == 1 ? 0.5 : -0.5) * sqrt(3.0) * base;
                            } else {
                                ovl += ovs * base;
                            }
                        }
                    } else if (c.e < H) {
                        hkey = ((uint32_t)c.e << 3) | ((ground ? 1u : 0u) << 2) | (uint32_t)(ovs + 1);
                    }
                    if (P.dump_mode && threadIdx.x < NT) {
                        // a binomial group emits each of its wall configurations c
                        const uint32_t nout = binc ? (1u << P.k) : 1u;
                        const uint32_t d0 = atomicAdd(P.dump.count, nout);
                        const uint64_t hh = config_hash(c, xs, C);
                        for (uint32_t q = 0; q < nout; ++q) {
                            const uint32_t di = d0 + q;
                            if (di >= P.dump.cap) break;
                            const uint32_t col = lab;
                            uint32_t sg = c.sign, cbq = c.cb;
                            double sc = (qubit ? sqrt(ldexp(1.0, -P.k)) : 1.0) * ae;
                            if (binc) {
                                cbq = q;
                                sg = (c.sign + __popc(q & c.cb)) & 1u;
                                sc *= apow(S, 2 * n * __popc(q));
                            }
                            double pr = (qubit && sg) ? -1.0 : 1.0, pim = 0.0;   // phase of the component
                            if (!qubit && sg) { pr = -0.5; pim = (sg == 1 ? 0.5 : -0.5) * sqrt(3.0); }
                            const double ar = __ldg(P.amp_re + col), ai = __ldg(P.amp_im + col);
                            P.dump.col[di] = col;
                            P.dump.bus[di] = cbq;
                            P.dump.hash[di] = hh;
                            P.dump.re[di] = (ar * pr - ai * pim) * sc;
                            P.dump.im[di] = (ar * pim + ai * pr) * sc;
                        }
                    }
                }
            }
            if (uni) {
                // integer histogram counts (shared-memory atomics; sums are order-free)
                if (hkey != 0xFFFFFFFFu && !binc) {
                    const uint32_t e = hkey >> 3;
                    atomicAdd(&hall[e], mc);
                    if ((hkey >> 2) & 1u) atomicAdd(&hemp[e], mc);
                    const int ovs = (int)(hkey & 3u) - 1;
                    if (ovs) atomicAdd(&hov[e], ovs);
                } else if (hkey != 0xFFFFFFFFu) {
                    // a binomial group: C(k, w) configurations at exponent e0 + 2n w;
                    // overlap (-1)^s0 K_w(|phi ^ b_out|) at the final epoch
                    const uint32_t e = hkey >> 3;
                    const int ovs = (int)(hkey & 3u) - 1;
                    for (int q = 0; q <= P.k; ++q) {
                        const uint32_t eb = e + (uint32_t)(2 * n * q);
                        if (eb >= (uint32_t)H) break;
                        const uint32_t cnt = (uint32_t)binom(P.k, q);
                        atomicAdd(&hall[eb], cnt);
                        if ((hkey >> 2) & 1u) atomicAdd(&hemp[eb], cnt);
                        if (ovs) {
                            const int kv = ovs * kraw(P.k, q, binm);
                            if (kv) atomicAdd(&hov[eb], kv);
                        }
                    }
                }
            }
            if (alive && !final_epoch && nent) S.anyent = 1u;
            put_entries((alive && !final_epoch) ? nent : 0u, pfc ? &pm : nullptr, c1, mcnt, uni ? c.e : 0, binc, w,
                        !uni, pwf, selk, selw, scr.selseg, wcur, lane, capfail);
            {
                const uint32_t flags = (binc ? kBinFlag : 0u) | (pfc ? kPFFlag : 0u);
                size_t dst = cbase + r;
                if (compact) {
                    uint32_t tot;
                    const uint32_t pre = block_scan_flag(alive, &tot, S);
                    dst = cbase + wr + pre;
                    wr += tot;
                }
                if (alive && !final_epoch) {
                    store_comp(scr, dst, c, xs, qubit, lab | flags, addr);
                    if (pfc) { pf_store(scr, dst, rec); S.pfnext = 1u; }
                }
            }
        }
        if (lane == 0) S.segn[warp] = min(wcur, scr.selseg);
        nsl = __reduce_add_sync(0xFFFFFFFFu, nsl);
        if (lane == 0 && nsl) atomicAdd(&S.wk[1], nsl);
        if (__any_sync(0xFFFFFFFFu, (n2p | nreg | nmem | noff) != 0u)) {
            n2p = __reduce_add_sync(0xFFFFFFFFu, n2p);
            nreg = __reduce_add_sync(0xFFFFFFFFu, nreg);
            nmem = __reduce_add_sync(0xFFFFFFFFu, nmem);
            noff = __reduce_add_sync(0xFFFFFFFFu, noff);
            if (lane == 0) {
                atomicAdd(&S.wk[4], n2p); atomicAdd(&S.wk[5], nreg);
                atomicAdd(&S.wk[6], nmem); atomicAdd(&S.wk[7], noff);
            }
        }
        if (threadIdx.x == 0) {
            if (lazy_pre) S.wk[2] += (uint32_t)P.D;
            else S.wk[3] += ncomp_pass;
        }
        if (__syncthreads_or(capfail) && threadIdx.x == 0) S.status = QRAM_E_CAP;
        __syncthreads();
        if (threadIdx.x == 0 && compact) S.ncomp = wr;
        if (threadIdx.x == 0 && !lazy_pre) S.haspf = S.pfnext;
        // No component with a non-empty mask: every weight went into both sums
        // alike, so Wemp = Wtot and no jump can fire; the sums are not needed
        // (the histograms are only cleared).
        const bool nodraw = !final_epoch && !lazy_pre && !S.anyent && (compact ? wr : ncomp) > 0u;
        if (nodraw) {
            for (int b = threadIdx.x; uni && b < H; b += NT)
                if (hall[b]) { hall[b] = 0; hemp[b] = 0; hov[b] = 0; }
            wsum = 1.0; wempty = 1.0;
        } else if (uni && !(lazy_pre && factored)) {
            // fold the histograms (and leave them zero for the next epoch)
            __syncthreads();
            for (int b = threadIdx.x; b < H; b += NT) {
                const uint32_t ca = hall[b];
                if (!ca) continue;
                const double ae = apow(S, b), a2 = ae * ae;
                wsum += (double)ca * a2;
                const uint32_t ce = final_epoch ? hemp[b] : ca - hemp[b];   // ground / empty mask
                if (ce) wempty += (double)ce * a2;
                const int co = hov[b];
                if (co) ovl += (double)co * ae;
                hall[b] = 0; hemp[b] = 0; hov[b] = 0;
            }
        }
        if (!nodraw) block_sum3(wsum, wempty, ovl, S, S.fW, S.fW, S.fO);
        // good branches of the eager form: closed-form weights before the
        // first jump (Eq. (21))
        double wgs = 0.0, ogs = 0.0;
        if (P.mode == kPruned && !jumped && !lazy && !depol && !heat && !nodraw) {
            const int sw = final_epoch ? T - 1 : s1 - 1;
            for (uint32_t b = threadIdx.x; b < (uint32_t)P.D; b += NT) {
                const uint32_t i = __ldg(P.addr + b);
                if ((S.badbits[i >> 5] >> (i & 31u)) & 1u) continue;
                if ((int)b == S.refcol) continue;
                const double ae = apow(S, good_exposure(P, b, sw));
                const double w2 = col_w2(P, b);
                wgs += w2 * ae * ae;
                if (final_epoch) ogs += w2 * ae;
            }
            double dummy = 0.0;
            block_sum3(wgs, ogs, dummy, S);
            wgs *= S.dn;
            ogs *= S.al;
        }
        const double Wtot = wsum + wgs, Wemp = wempty + wgs;
        if (final_epoch) {
            const double ov_all = ovl + ogs;
            double ov_im = 0.0;                       // imaginary part (qutrit phases of depolarizing faults)
            if (depol && !qubit) ov_im = block_sum(ovi, S.redA, S);
            const double ov2 = ov_all * ov_all + ov_im * ov_im;
            if (threadIdx.x == 0) {
                const double uf = uniform53(P.seed, 0, 3u, traj);
                const bool ground = Wemp > uf * Wtot;
                qram_result_t R;
                R.fidelity = (ground && Wemp > 0.0) ? ov2 / Wemp : 0.0;
                R.fidelity_unsampled = Wtot > 0.0 ? ov2 / Wtot : 0.0;
                R.p_ground = Wtot > 0.0 ? Wemp / Wtot : 0.0;
                R.bad = S.nbad;
                R.ref = S.refcol;
                R.ncand = S.ncand;
                R.explicit_comps = ncomp0;
                R.jumps = (uint16_t)jumps;
                R.first_jump_slice = (uint16_t)first_jump;
                R.jump_sites = (uint16_t)jump_sites;
                R.q_ground = ground ? 1 : 0;
                R.status = (uint8_t)S.status;
                if (P.out) P.out[t] = R;
                if (P.ctr)
                    for (int q = 0; q < 8; ++q) atomicAdd(P.ctr + q, (unsigned long long)S.wk[q]);
                if (P.dump_mode) {
                    P.dump.scal[0] = Wtot;
                    P.dump.scal[1] = jumped ? 1.0 : 0.0;
                    P.dump.scal[2] = (depol || heat) ? 1.0 : 0.0; // every branch explicit: nothing to predict
                    P.dump.scal[3] = lazy ? 1.0 : 0.0;            // no branch explicit before a jump
                }
            }
            __syncthreads();
            return;
        }
        // ---- 5. joint draw at slice s1 (Theorem 3 with Eq. (21) weights) ----
        const double u = uniform53(P.seed, (uint32_t)s1, 2u, traj);
        double tgt = u * Wtot;
        int nsel = 0;
        if (!(Wemp > tgt) && S.status == QRAM_OK && lazy_pre) {
            // a jump may fire: give the configurations with a non-empty mask
            // explicit state (after the gates of s1, K0 through s1 - 1) and
            // the compact list of (first element, size, weight) the descent reads
            const uint32_t pos = S.cl2 & P.orbit.occ[s1];
            // before the first wall no data qubit is in the tree (no data
            // hits): one merged component per branch stands for its 2^k
            // configurations
            if (mergeable && s1 <= 2 * n) mlog = P.k;
            // from slice sU on every data qubit is in the bus: one binomial
            // group per branch (its configurations are on the noiseless orbit:
            // exponents E0 + 2n|c|, signs c.(j ^ d), Lemma 1)
            const bool mbin = binok && s1 >= sU;
            // in between, one component in product form per branch
            const bool mpf = pfok && mlog == 0 && !mbin;
            const uint32_t ncw = (qubit && mlog == 0 && !mbin && !mpf) ? (1u << P.k) : 1u;
            const double wmul = (double)(1u << mlog) * (mbin ? S.bw : 1.0);
            uint32_t base = 0;
            bool capfail = false;
            for (uint32_t b0 = 0; b0 < (uint32_t)P.D; b0 += NT) {
                const uint32_t b = b0 + threadIdx.x;
                uint32_t cnt = 0, tm = 0, i = 0, j = 0, d = 0;
                bool all = false;
                if (b < (uint32_t)P.D) {
                    i = __ldg(P.addr + b); j = __ldg(P.bus + b); d = __ldg(P.mem + i);
                    if ((S.hitbits[i >> 5] >> (i & 31u)) & 1u) tm = orbit_hits(P, S.candbits, pos, s1, i, j, d, all);
                    cnt = all ? ncw : (tm ? ncw - (ncw >> __popc(tm)) : 0u);
                    if ((mlog > 0 || mbin) && tm) { capfail = true; cnt = 0; }   // (no data qubit in the tree then)
                }
                uint32_t tot;
                const uint32_t pre = block_scan_count(cnt, &tot, S);
                if (base + tot > scr.ecap) { capfail = true; break; }
                uint32_t r = base + pre;
                // (qubit: this epoch's nibble tables hold the exposure at s1 - 1)
                const int E0 = !cnt ? 0
                             : qubit ? S.etab[0][i & 15u] + S.etab[1][(i >> 4) & 15u] + S.etab[2][(i >> 8) & 15u] +
                                           S.etab[3][(i >> 12) & 15u]
                                     : good_exposure(P, b, s1 - 1);
                const double w2 = cnt ? (uni ? w2u : col_w2(P, b) * k2) : 0.0;
                const Ctx C = make_ctx(P.enc, n, P.mem, i);
                for (uint32_t cw = 0; cw < ncw; ++cw) {
                    const bool take = cnt && (mpf || all || (cw & tm));
                    uint32_t c1 = 0, mcnt = 0, nent = 0;
                    int ce = 0;
                    double w = 0.0, pwf = 0.0;
                    PFMasks pm;
                    if (take) {
                        CompR c = orbit_state(P, s1, i, cw, j, d);
                        c.e = E0 + (qubit ? data_exposure(P, cw, s1 - 1) : 0);
                        if (mbin) c.cb = (j ^ (d & P.orbit.fetched[s1])) & kmask;   // phi of the group
                        uint32_t rec[8];
                        if (mpf) {
                            // the address part is configuration 0; data qubit t on its
                            // orbit position (or bus slot), exposed for its window so
                            // far, phase bit j_t plus its fetched memory bit
                            for (int t = 0; t < 8; ++t) rec[t] = 0u;
                            const uint32_t fm = P.orbit.fetched[s1], bm = P.orbit.bus[s1];
                            for (int t = 0; t < P.k; ++t) {
                                const uint32_t m = (uint32_t)ov(2 * n + 2 * t + 1, 4 * n + 2 * t, s1 - 1);
                                const uint32_t ph = ((j >> t) ^ ((fm >> t) & (d >> t))) & 1u;
                                rec[t] = kPFree | (ph ? kPPh : 0u) | (m << 16) | kPBus | (uint32_t)t;
                                const int bb = P.orbit.dpos[s1][t];
                                if (!((bm >> t) & 1u) && bb >= 0)
                                    rec[t] = kPFree | (ph ? kPPh : 0u) | (m << 16) |
                                             (2u * path_node(i, n, bb >> 1) + (uint32_t)(bb & 1));
                            }
                            pf_store(scr, cbase + r, rec);
                        }
                        store_comp(scr, cbase + r, c, nullptr, qubit, b | (mbin ? kBinFlag : 0u) | (mpf ? kPFFlag : 0u), i);
                        ++r;
                        c1 = mask_first(c, nullptr, C, S.candbits, S.cl2, mcnt);
                        ce = c.e;
                        nent = 1;
                        const int etop = mpf ? pf_etop(rec, P.k, c.e) : c.e + (mbin ? 2 * n * P.k : 0);
                        if (etop >= 4096 || (uni && etop >= H)) capfail = true;  // the key holds 12 bits of e
                        if (mpf) {
                            pf_masks(rec, P.k, c.e, S.candbits, S.powlo, S.powhi, pm);
                            pwf = uni ? 1.0 : w2;
                            nent = (1u << pm.ntc) - (mcnt == 0 ? 1u : 0u);
                        } else if (!uni) {
                            const double ae = apow(S, c.e);
                            w = w2 * ae * ae * wmul;
                        }
                    }
                    put_entries(nent, mpf ? &pm : nullptr, c1, mcnt, uni ? ce : 0, mbin, w, !uni, pwf, selk, selw,
                                scr.selseg, wcur, lane, capfail);
                }
                base += tot;
            }
            if (lane == 0) S.segn[warp] = min(wcur, scr.selseg);
            if (__syncthreads_or(capfail) && threadIdx.x == 0) S.status = QRAM_E_CAP;
            if (threadIdx.x == 0) { S.ncomp = base; S.haspf = (mpf && base > 0) ? 1u : 0u; }
            __syncthreads();
        }
        if (!(Wemp > tgt) && S.status == QRAM_OK) {
            // descent over the canonical order; O = weight before the subtree
            double O = Wemp;
            const uint32_t cb0 = S.slice_off[s1], ncodes = 2u * (S.slice_off[s1 + 1] - cb0);
            __shared__ uint32_t pref[kMaxJ];
            // level 0 on the compact list: first element x with O + F(x) > tgt,
            // F(x) = weight of components whose first element is <= x
            int start = 0;
            bool decided = false;
            {
                const uint32_t *sk0 = scr.selk + slot * NW * (size_t)scr.selseg;
                const double *sw0 = scr.selw + slot * NW * (size_t)scr.selseg;
                // block sum of the weights of the selected entries; equal
                // magnitudes count their exponents in the integer histogram
                // and fold its non-empty bins (FP64 work per bin, not per
                // entry: a first jump can select tens of thousands)
                auto Fsum = [&](uint32_t cmax, uint32_t ceq, bool eq_only_single, int *multi) {
                    double f = 0.0;
                    int mm = 0;
                    for (uint32_t q = 0; q < NW; ++q) {
                        const uint32_t *sk = sk0 + q * (size_t)scr.selseg;
                        const double *sw = sw0 + q * (size_t)scr.selseg;
                        for (uint32_t e = threadIdx.x; e < S.segn[q]; e += NT) {
                            const uint32_t kv = sk[e], code = kv & 0xFFFFu;
                            const bool in = eq_only_single ? code == ceq && ((kv >> 16) & 7u) == 1u : code <= cmax;
                            if (eq_only_single && code == ceq && !in) mm = 1;
                            if (in) {
                                const uint32_t ex = kv >> 20;
                                if (uni && ex != kPFKey) {
                                    if (!((kv >> 19) & 1u)) {
                                        if (ex < (uint32_t)H) atomicAdd(&hall[ex], 1u);
                                    } else {                   // a binomial group
                                        for (int q = 0; q <= P.k; ++q) {
                                            const uint32_t eb = ex + (uint32_t)(2 * n * q);
                                            if (eb < (uint32_t)H) atomicAdd(&hall[eb], (uint32_t)binom(P.k, q));
                                        }
                                    }
                                } else {
                                    f += sw[e];
                                }
                            }
                        }
                    }
                    if (uni) {
                        __syncthreads();
                        for (int b = (int)threadIdx.x; b < H; b += NT) {
                            const uint32_t cnt = hall[b];
                            if (!cnt) continue;
                            const double ae = apow(S, b);
                            f += (double)cnt * (ae * ae);
                            hall[b] = 0;
                        }
                    }
                    if (multi) *multi = mm;
                    return block_sum(f, S.redA, S) * (uni ? w2u * (double)(1u << mlog) : 1.0);
                };
                uint32_t lo = 0, hi = ncodes;
                double Flo = 0.0;
                // A short list (at most 8 NT entries) is searched directly: each
                // entry's first code is turned once into its index among the
                // slice's codes (the candidate sites staged, ascending, in the
                // zero hemp area) and its weight into FP64, in place in the
                // list; every step of the search is then a compare-and-add per
                // entry and one block sum.  Longer lists (a first jump of many
                // branches) keep the histogram sums.
                const uint32_t ncs = ncodes / 2u;
                uint32_t tot = 0;
                for (uint32_t q = 0; q < NW; ++q) tot += S.segn[q];
                const bool direct = tot <= 8u * NT && ncs <= (uint32_t)P.hist_pad && ncodes / 16u + 2u <= (uint32_t)P.hist_pad;
                uint32_t *skw = scr.selk + slot * NW * (size_t)scr.selseg;
                double *sww = scr.selw + slot * NW * (size_t)scr.selseg;
                auto each_entry = [&](auto &&fn) {
                    for (uint32_t q = 0; q < NW; ++q) {
                        const uint32_t nq = S.segn[q];
                        for (uint32_t e = threadIdx.x; e < nq; e += NT) fn(q * (size_t)scr.selseg + e);
                    }
                };
                const double fsc = uni ? w2u * (double)(1u << mlog) : 1.0;
                if (direct) {
                    for (uint32_t c = threadIdx.x; c < ncs; c += NT) hemp[c] = cand[cb0 + c] & 0xFFFFu;
                    __syncthreads();
                    each_entry([&](size_t at) {
                        const uint32_t kv = skw[at], code = kv & 0xFFFFu, site = code >> 1, ex = kv >> 20;
                        uint32_t a0 = 0, a1 = ncs;
                        while (a0 < a1) {
                            const uint32_t m = (a0 + a1) >> 1;
                            if (hemp[m] < site) a0 = m + 1; else a1 = m;
                        }
                        double w;
                        if (!uni || ex == kPFKey) {
                            w = sww[at];
                        } else {
                            const double ae = apow(S, (int)ex);
                            w = ae * ae * (((kv >> 19) & 1u) ? S.bw : 1.0);       // a binomial group: (1 + a^(4n))^k
                        }
                        const uint32_t ci = 2u * a0 + (code & 1u);
                        skw[at] = ci | (((kv >> 16) & 7u) << 16);
                        sww[at] = w;
                        atomicOr(&hov[ci >> 5], 1u << (ci & 31u));     // the code occurs
                    });
                    __syncthreads();
                    for (uint32_t c = threadIdx.x; c < ncs; c += NT) hemp[c] = 0u;
                    // F changes only at codes that occur: their ascending list
                    // is what the search visits (the bitmap area doubles as the
                    // block sums' partials, so the list sits in static memory)
                    if (threadIdx.x == 0) {
                        uint32_t m = 0;
                        for (uint32_t wd = 0; wd < (ncodes + 31u) / 32u; ++wd)
                            for (uint32_t bits = (uint32_t)hov[wd]; bits; bits &= bits - 1u) {
                                if (m < 128u) S.plist[m] = (uint16_t)(32u * wd + (uint32_t)(__ffs(bits) - 1));
                                ++m;
                            }
                        S.npres = m;
                    }
                    __syncthreads();
                    for (uint32_t w = threadIdx.x; w < (ncodes + 31u) / 32u; w += NT) hov[w] = 0;
                    __syncthreads();
                }
                auto Fdir = [&](uint32_t ximax) {
                    double f = 0.0;
                    each_entry([&](size_t at) { if ((skw[at] & 0xFFFFu) <= ximax) f += sww[at]; });
                    return block_sum(f, S.redA, S) * fsc;
                };
                if (direct && S.npres <= 128u) {
                    const uint32_t np = S.npres;
                    uint32_t a0 = 0, a1 = np;
                    while (a0 < a1) {
                        const uint32_t mid = (a0 + a1) >> 1;
                        const double f = Fdir((uint32_t)S.plist[mid]);
                        if (O + f > tgt) a1 = mid;
                        else { a0 = mid + 1; Flo = f; }
                    }
                    lo = a0 < np ? (uint32_t)S.plist[a0] : ncodes;
                } else if (direct) {
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        const double f = Fdir(mid);
                        if (O + f > tgt) hi = mid;
                        else { lo = mid + 1; Flo = f; }
                    }
                } else {
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        const uint32_t cmid = 2u * (cand[cb0 + (mid >> 1)] & 0xFFFFu) + (mid & 1u);
                        const double f = Fsum(cmid, 0, false, nullptr);
                        if (O + f > tgt) hi = mid;
                        else { lo = mid + 1; Flo = f; }
                    }
                }
                if (lo < ncodes) {
                    const uint32_t code = 2u * (cand[cb0 + (lo >> 1)] & 0xFFFFu) + (lo & 1u);
                    O += Flo;
                    int mm = 0;
                    double wex;
                    if (direct) {
                        double f = 0.0;
                        each_entry([&](size_t at) {
                            const uint32_t kv = skw[at];
                            if ((kv & 0xFFFFu) != lo) return;
                            if (((kv >> 16) & 7u) == 1u) f += sww[at]; else mm = 1;
                        });
                        wex = block_sum(f, S.redA, S) * fsc;
                    } else {
                        wex = Fsum(0, code, true, &mm);
                    }
                    const int multi = __syncthreads_or(mm);
                    if (threadIdx.x == 0) pref[0] = code;
                    __syncthreads();
                    nsel = 1;
                    if (!multi || O + wex > tgt) decided = true;       // J = [code]
                    else start = 1;                                     // longer masks: general descent
                }
            }
            // fn(q, weight) for each mask of component r: q is mask_query's
            // answer for the prefix pref[0..level); a component in product
            // form has one mask per subset of its data qubits at candidates
            auto masks_of = [&](uint32_t r, int level, auto &&fn) {
                CompR c; alignas(16) uint16_t xs[kXcap]; uint32_t lab, addr;
                const uint4 rv = scr.cs[cbase + r];
                unpack(rv, qubit, c, lab, addr);
                if (c.nexc) load_exc(scr, cbase + r, c.nexc, xs);
                const Ctx C = make_ctx(P.enc, n, P.mem, addr);
                const double wf = uni ? w2u : col_w2(P, lab) * k2;
                if (rv.w & kPFFlag) {
                    uint32_t rec[8];
                    PFMasks pm;
                    pf_load(scr, cbase + r, rec);
                    pf_masks(rec, P.k, c.e, S.candbits, S.powlo, S.powhi, pm);
                    for (uint32_t sb = 0; sb < (1u << pm.ntc); ++sb) {
                        uint32_t xc[kMaxK];
                        int nx = 0;
                        double wt = wf * pm.base;
                        for (uint32_t q = 0; q < pm.ntc; ++q)
                            if ((sb >> q) & 1u) { xc[nx++] = pm.code[q]; wt *= pm.f[q]; }
                        fn(mask_query(c, xs, C, S.candbits, pref, level, xc, nx), wt);
                    }
                    return;
                }
                const long long q = heat ? mask_query_heat(c, xs, C, cand, pev, S.slice_off[s1], S.slice_off[s1 + 1], pref, level)
                                         : mask_query(c, xs, C, S.candbits, pref, level);
                const double ae = apow(S, c.e);
                fn(q, wf * (double)(1u << mlog) * ae * ae * ((rv.w & kBinFlag) ? S.bw : 1.0));
            };
            for (int level = start; level < kMaxJ && !decided; ++level) {
                // weight of components whose mask equals the prefix exactly
                if (level > 0) {
                    double we = 0.0;
                    for (uint32_t r = threadIdx.x; r < S.ncomp; r += NT)
                        masks_of(r, level, [&](long long q, double wt) { if (q == -1) we += wt; });
                    we = block_sum(we, S.redA, S);
                    if (O + we > tgt) break;                  // J = prefix
                    O += we;
                }
                // F(x): weight with next code <= code(x); find first x with O + F(x) > tgt
                uint32_t lo = 0, hi = ncodes;                // answer in [lo, hi]; hi = none
                double Flo = 0.0;                            // F(lo - 1)
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    const uint32_t cmid = 2u * (cand[cb0 + (mid >> 1)] & 0xFFFFu) + (mid & 1u);
                    double f = 0.0;
                    for (uint32_t r = threadIdx.x; r < S.ncomp; r += NT)
                        masks_of(r, level, [&](long long q, double wt) { if (q >= 0 && (uint32_t)q <= cmid) f += wt; });
                    f = block_sum(f, S.redA, S);
                    if (O + f > tgt) hi = mid;
                    else { lo = mid + 1; Flo = f; }
                }
                if (lo >= ncodes) {
                    // rounding left the target above the total: take the last
                    // group with weight (the oracle's rule); descend on the largest code
                    uint32_t best = 0xFFFFFFFFu;
                    for (uint32_t r = threadIdx.x; r < S.ncomp; r += NT)
                        masks_of(r, level, [&](long long q, double) {
                            if (q >= 0 && (best == 0xFFFFFFFFu || (uint32_t)q > best)) best = (uint32_t)q;
                        });
                    __shared__ uint32_t sbest;
                    if (threadIdx.x == 0) sbest = 0u;
                    __syncthreads();
                    if (best != 0xFFFFFFFFu) atomicMax(&sbest, best + 1u);
                    __syncthreads();
                    const uint32_t sb = sbest;
                    __syncthreads();
                    if (sb == 0u) break;                                // mask == prefix
                    const uint32_t code = sb - 1u;
                    if (threadIdx.x == 0) pref[level] = code;
                    __syncthreads();
                    tgt = O + 1e308;                                    // keep taking the last group
                    nsel = level + 1;
                    continue;
                }
                const uint32_t code = 2u * (cand[cb0 + (lo >> 1)] & 0xFFFFu) + (lo & 1u);
                if (threadIdx.x == 0) pref[level] = code;
                __syncthreads();
                O += Flo;
                nsel = level + 1;
            }
            if (threadIdx.x == 0) {
                for (int j = 0; j < nsel; ++j) S.J[j] = pref[j];
            }
        }
        if (threadIdx.x == 0) {
            S.nJ = nsel;
            if (lazy_pre && nsel == 0) { S.ncomp = 0; S.haspf = 0u; }   // no jump: the branches stay implicit
        }
        if (lazy_pre && nsel == 0) mlog = 0;
        __syncthreads();
        if (nsel > 0) {
            if (!jumped) first_jump = (uint32_t)s1;
            ++jumps;
            jump_sites += (uint32_t)nsel;
            // Relevance after a jump.  Every survivor held all of J on its
            // address path; an item can only leave that path below a damaged
            // router and only into that router's subtree, and it can only
            // leave a subtree through its root.  So all later excitations lie
            // on the path to r = LCA(J, earlier roots) or inside subtree(r):
            // candidates elsewhere leave J empty and need no draw.
            if (threadIdx.x == 0) {
                uint32_t r = jumped ? S.region : (S.J[0] >> 2);
                for (int q = 0; q < nsel; ++q) r = tree_lca(r, S.J[q] >> 2);
                S.region = r;
                S.syncmask[4] = S.syncmask[5] = S.syncmask[6] = S.syncmask[7] = 0;
            }
            jumped = true;
            __syncthreads();
            const uint32_t r = S.region;
            for (uint32_t c = S.slice_off[s1 + 1] + threadIdx.x; c < S.slice_off[T]; c += NT) {
                const uint32_t u = (cand[c] & 0xFFFFu) >> 1, sc = cand[c] >> 16;
                if (depol || heat || tree_related(u, r)) atomicOr(&S.syncmask[4 + (sc >> 5)], 1u << (sc & 31u));
            }
        }
        // clear the candidate bitmaps of s1 (the hit bitmap word by word: a
        // candidate near the root covers most of it)
        for (uint32_t c = S.slice_off[s1] + threadIdx.x; c < S.slice_off[s1 + 1]; c += NT) {
            const uint32_t site = cand[c] & 0xFFFFu;
            atomicAnd(&S.candbits[site >> 5], ~(1u << (site & 31u)));
        }
        if (lazy_pre)
            for (uint32_t wd = threadIdx.x; wd < ((1u << n) + 31u) / 32u; wd += NT) S.hitbits[wd] = 0u;
        if (threadIdx.x == 0 && (clock64() - S.t_start > kCycleBudget || s1 <= s_prev)) S.status = QRAM_E_TIMEOUT;
        __syncthreads();
        s_prev = s1;
    }
}

// DEPOL: compiled with the depolarizing faults (a launch with eps > 0);
// without, the event code is absent from the hot loop
template <int NT, int MINB, bool DEPOL>
__global__ void __launch_bounds__(NT, MINB) traj_kernel(const __grid_constant__ Params P) {
    __shared__ Smem<NT> S;
    // 3 exponent histograms of hist_pad bins, or the partials of a block sum;
    // kept zero between uses
    extern __shared__ __align__(16) uint32_t dyn_hist[];
    for (uint32_t b = threadIdx.x; b < dyn_words(P.n, P.k, NT); b += NT) dyn_hist[b] = 0;
    if (threadIdx.x == 0) S.part = reinterpret_cast<double *>(dyn_hist);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t w = atomicAdd(P.work, 1u);
            S.t = (int)((P.perm && w < P.ntraj) ? __ldg(P.perm + w) : w);   // longest first (launch_order)
        }
        __syncthreads();
        const uint32_t t = (uint32_t)S.t;
        __syncthreads();
        if (t >= P.ntraj) break;
        run_one<NT, DEPOL>(P, S, t, dyn_hist);
        __syncthreads();
    }
}

// Mixed persistent launch: one work-stealing loop over the trajectories of
// several problems.  A CTA maps the global trajectory index to its problem,
// copies that problem's Params from device memory into shared memory when
// the problem changes, and runs the same per-trajectory code as traj_kernel
// (damping only: the depolarizing variant is not instantiated here).  Every
// problem's scratch holds at least gridDim.x slots.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) traj_kernel_multi(const __grid_constant__ MultiParams MP) {
    __shared__ Smem<NT> S;
    __shared__ __align__(16) Params Ps;
    extern __shared__ __align__(16) uint32_t dyn_hist[];
    for (uint32_t b = threadIdx.x; b < MP.dyn_words; b += NT) dyn_hist[b] = 0;
    if (threadIdx.x == 0) S.part = reinterpret_cast<double *>(dyn_hist);
    __syncthreads();
    const uint32_t total = MP.start[MP.nprob];
    int cur = -1;                                   // problem whose Params are in Ps (same in every thread)
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t w = atomicAdd(MP.work, 1u);
            S.t = (int)((MP.perm && w < total) ? __ldg(MP.perm + w) : w);   // longest first (launch_order_multi)
        }
        __syncthreads();
        const uint32_t t = (uint32_t)S.t;
        __syncthreads();
        if (t >= total) break;
        int p = 0;
        while (p + 1 < (int)MP.nprob && t >= MP.start[p + 1]) ++p;
        if (p != cur) {
            static_assert(sizeof(Params) % 8 == 0, "Params copy in 8-byte words");
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(MP.probs + p);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(&Ps);
            for (uint32_t w = threadIdx.x; w < sizeof(Params) / 8; w += NT) dst[w] = src[w];
            cur = p;
            __syncthreads();
        }
        run_one<NT, false>(Ps, S, t - MP.start[p], dyn_hist);
        __syncthreads();
    }
}

template <int NT, int MINB>
static cudaError_t launch_multi_variant(const MultiParams &mp, int grid, size_t dyn, cudaStream_t s,
                                        bool occupancy_only, int *blocks) {
    cudaError_t e = cudaFuncSetAttribute(traj_kernel_multi<NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(3 * kHistMax * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    if (occupancy_only)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, traj_kernel_multi<NT, MINB>, NT, dyn);
    traj_kernel_multi<NT, MINB><<<grid, NT, dyn, s>>>(mp);
    return cudaGetLastError();
}

static cudaError_t dispatch_multi(int threads, const MultiParams &mp, int grid, size_t dyn, cudaStream_t s, bool occ,
                                  int *blocks) {
    switch (threads) {
    case 128: return launch_multi_variant<128, 8>(mp, grid, dyn, s, occ, blocks);
    case 256: return launch_multi_variant<256, 4>(mp, grid, dyn, s, occ, blocks);
    case 512: return launch_multi_variant<512, 2>(mp, grid, dyn, s, occ, blocks);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_trajectories_multi(const MultiParams &mp, int grid, int threads, size_t dyn, cudaStream_t s) {
    return dispatch_multi(threads, mp, grid, dyn, s, false, nullptr);
}

int kernel_blocks_per_sm_multi(int threads, size_t dyn) {
    int b = 0;
    if (dispatch_multi(threads, MultiParams{}, 0, dyn, nullptr, true, &b) != cudaSuccess) { cudaGetLastError(); return 0; }
    return b;
}

// launch variants (threads per CTA, minimum resident CTAs for the register cap)
template <int NT, int MINB, bool DEPOL>
static cudaError_t launch_variant(const Params &p, int grid, size_t dyn, cudaStream_t s, bool occupancy_only, int *blocks) {
    // static + dynamic shared memory can exceed 48 KB: opt in
    cudaError_t e = cudaFuncSetAttribute(traj_kernel<NT, MINB, DEPOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(3 * kHistMax * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    if (occupancy_only)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, traj_kernel<NT, MINB, DEPOL>, NT, dyn);
    traj_kernel<NT, MINB, DEPOL><<<grid, NT, dyn, s>>>(p);
    return cudaGetLastError();
}

static cudaError_t dispatch(int threads, const Params &p, int grid, size_t dyn, cudaStream_t s, bool occ, int *blocks) {
    const bool depol = p.eps > 0.0 || p.eps_gamma;
    switch (threads) {
    case 128: return depol ? launch_variant<128, 8, true>(p, grid, dyn, s, occ, blocks)
                           : launch_variant<128, 8, false>(p, grid, dyn, s, occ, blocks);
    case 256: return depol ? launch_variant<256, 4, true>(p, grid, dyn, s, occ, blocks)
                           : launch_variant<256, 4, false>(p, grid, dyn, s, occ, blocks);
    case 512: return depol ? launch_variant<512, 2, true>(p, grid, dyn, s, occ, blocks)
                           : launch_variant<512, 2, false>(p, grid, dyn, s, occ, blocks);
    case 1024: return depol ? launch_variant<1024, 1, true>(p, grid, dyn, s, occ, blocks)
                            : launch_variant<1024, 1, false>(p, grid, dyn, s, occ, blocks);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_trajectories(const Params &p, int grid, int threads, size_t dyn, cudaStream_t s) {
    return dispatch(threads, p, grid, dyn, s, false, nullptr);
}

int hist_pad(int n, int k) {
    const int H = (2 * n + k) * (6 * n + 2 * k - 1) + 1;
    return (H + 31) & ~31;
}

size_t dyn_smem_bytes(int n, int k, int threads) { return (size_t)dyn_words(n, k, threads) * sizeof(uint32_t); }

bool valid_threads(int threads) { return threads == 128 || threads == 256 || threads == 512 || threads == 1024; }

int kernel_threads() { return 256; }

int kernel_blocks_per_sm(int threads, size_t dyn) {
    int b = 0;
    if (dispatch(threads, Params{}, 0, dyn, nullptr, true, &b) != cudaSuccess) { cudaGetLastError(); return 0; }
    return b;
}

// ---------------------------------------------------------------------------
// ensemble mean / standard error in a fixed order (one CTA)
__global__ void __launch_bounds__(256) fidelity_kernel(const qram_result_t *res, uint32_t ntraj, double *out2) {
    __shared__ double ra[8], rb[8];
    double s = 0.0, q = 0.0;
    for (uint32_t t = threadIdx.x; t < ntraj; t += 256) { const double f = res[t].fidelity; s += f; q += f * f; }
    s = warp_sum(s); q = warp_sum(q);
    if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = s; rb[threadIdx.x >> 5] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S1 = 0.0, S2 = 0.0;
        for (int i = 0; i < 8; ++i) { S1 += ra[i]; S2 += rb[i]; }
        const double m = ntraj ? S1 / ntraj : 0.0;
        double var = ntraj > 1 ? (S2 - S1 * m) / (ntraj - 1) : 0.0;
        if (var < 0) var = 0;
        out2[0] = m;
        out2[1] = ntraj ? sqrt(var / ntraj) : 0.0;
    }
}

// |c|^2 * 2^-k if every input column has the same squared magnitude (bitwise),
// else 0: lets the trajectory kernel sum weights as integer exponent histograms.
__global__ void uniform_weight_kernel(const double *re, const double *im, int D, int qubit_k, double *out) {
    __shared__ int diff;
    if (threadIdx.x == 0) diff = 0;
    __syncthreads();
    const double w0 = re[0] * re[0] + im[0] * im[0];
    for (int b = threadIdx.x; b < D; b += blockDim.x) {
        const double w = re[b] * re[b] + im[b] * im[b];
        if (w != w0) diff = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) *out = (diff || !(w0 > 0.0)) ? 0.0 : w0 * ldexp(1.0, -qubit_k);
}

cudaError_t launch_uniform_weight(const double *re, const double *im, int D, int qubit_k, double *out, cudaStream_t s) {
    uniform_weight_kernel<<<1, 256, 0, s>>>(re, im, D, qubit_k, out);
    return cudaGetLastError();
}

cudaError_t launch_fidelity(const qram_result_t *res, uint32_t ntraj, double *out2, cudaStream_t s) {
    fidelity_kernel<<<1, 256, 0, s>>>(res, ntraj, out2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launch order, longest first.  Trajectories differ in cost by orders of
// magnitude: one whose first jump hits a router near the root while the
// address is loaded keeps thousands of branches explicit for most of the
// schedule.  Handing the expensive ones out first keeps a launch from ending
// on one of them started late.  Results do not depend on the order.
//
// Cost score of a trajectory: its damping candidates (the same fault stream
// as the trajectory kernel, regenerated) weighted by what a jump there would
// leave explicit, sum over candidates (s, q) of 2^(n - 2L) (T - s), L the
// layer of q: a jump on a layer-L router takes about 2^(n-L) branches out
// of the closed form with probability about 2^-L, for the T - s slices
// left.  Zero without candidates; -1 for a rate the trajectory rejects.
__device__ float traj_score(const Params &P, uint32_t t, uint64_t *gq, uint32_t lane) {
    const double gamma = P.gamma[t];
    if (!(gamma >= 0.0 && gamma < 1.0 && gamma < P.gamma_lim)) return -1.0f;
    const uint64_t thr = (uint64_t)__double2ull_rz(gamma * 18446744073709551616.0);
    if (thr == 0) return 0.0f;
    __syncwarp();
    if (lane == 0) {
        gq[0] = 0ull - thr;
        for (int m = 0; m + 1 < kGapBits; ++m) gq[m + 1] = __umul64hi(gq[m], gq[m]);
    }
    __syncwarp();
    const uint64_t traj = (P.traj0_dev ? *P.traj0_dev : P.traj0) + t;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    const uint32_t tl = (uint32_t)traj, th = (uint32_t)(traj >> 32);
    const uint32_t M = 2u * (uint32_t)P.nodes, X = (uint32_t)(P.T - 1) * M;
    const uint32_t nblk = (X + kGapBlock - 1) / kGapBlock;
    float sc = 0.0f;
    for (uint32_t g = lane; g < nblk; g += 32) {
        uint32_t pos = g * kGapBlock;
        const uint32_t end = min(pos + kGapBlock, X);
        uint32_t o0 = 0, o1 = 0, o2 = 0, o3 = 0;
        for (uint32_t r = 0;; ++r) {
            if ((r & 1u) == 0) {
                o0 = g; o1 = (r >> 1) | (1u << 24); o2 = tl; o3 = th;
                philox(o0, o1, o2, o3, k0, k1);
            }
            const uint64_t u = (r & 1u) ? ((uint64_t)o2 | ((uint64_t)o3 << 32)) : ((uint64_t)o0 | ((uint64_t)o1 << 32));
            uint64_t acc = ~0ull;
            uint32_t G = 0;
            for (int m = kGapBits - 1; m >= 0; --m) {
                const uint64_t v = __umul64hi(acc, gq[m]);
                if (v > u) { acc = v; G += 1u << m; }
            }
            if (G >= end - pos) break;
            pos += G;
            const int s = 1 + (int)(pos / M), L = layer_of((pos % M) >> 1);
            sc += ldexpf((float)(P.T - s), P.n - 2 * L);
            ++pos;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xFFFFFFFFu, sc, o);
    return sc;
}

// one warp per trajectory: score[i] of trajectory i of one problem (Params
// by value) or of the concatenated ranges of a mixed launch (table on the
// device)
__global__ void __launch_bounds__(256) score_kernel(const __grid_constant__ Params P, uint32_t n, float *score) {
    __shared__ uint64_t gq[8][kGapBits];
    const uint32_t lane = threadIdx.x & 31u, wi = threadIdx.x >> 5;
    for (uint64_t i = (uint64_t)blockIdx.x * 8 + wi; i < n; i += (uint64_t)gridDim.x * 8) {
        const float sc = traj_score(P, (uint32_t)i, gq[wi], lane);
        if (lane == 0) score[i] = sc;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) score_kernel_multi(const __grid_constant__ MultiParams MP, float *score) {
    __shared__ uint64_t gq[8][kGapBits];
    const uint32_t lane = threadIdx.x & 31u, wi = threadIdx.x >> 5;
    const uint32_t n = MP.start[MP.nprob];
    for (uint64_t i = (uint64_t)blockIdx.x * 8 + wi; i < n; i += (uint64_t)gridDim.x * 8) {
        uint32_t p = 0;
        while (p + 1 < MP.nprob && i >= MP.start[p + 1]) ++p;
        const float sc = traj_score(MP.probs[p], (uint32_t)i - MP.start[p], gq[wi], lane);
        if (lane == 0) score[i] = sc;
        __syncwarp();
    }
}

// Bucket of a score: quarter octaves below the key of an upper estimate
// (the exponent and two leading mantissa bits of a positive double grow
// with its value), highest first; no candidates next to last; rejected
// rates (nothing to evolve) last.
__device__ __forceinline__ int order_key(double x) {
    return (int)((unsigned long long)__double_as_longlong(x) >> 50);
}
struct ScoreKey {
    const float *score;
    int ktop;
    __device__ uint32_t operator()(uint32_t i) const {
        const float x = score[i];
        if (x > 0.0f) return (uint32_t)min(max(ktop - order_key((double)x), 0), kOrderBuckets - 2);
        return x == 0.0f ? kOrderBuckets - 2u : kOrderBuckets - 1u;
    }
};

// Counting sort of the indices 0 .. n-1 by bucket into perm (one CTA;
// shared-memory counts aggregated per warp over lanes of equal bucket);
// any order inside a bucket.
template <class Key>
__global__ void __launch_bounds__(1024) order_kernel(const __grid_constant__ Key key, uint32_t n, uint32_t *perm) {
    __shared__ uint32_t cnt[kOrderBuckets];
    const uint32_t lane = threadIdx.x & 31u;
    if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0u;
    __syncthreads();
    for (uint64_t b0 = 0; b0 < n; b0 += blockDim.x) {             // every warp runs every round
        const uint64_t i = b0 + threadIdx.x;
        const uint32_t b = i < n ? key((uint32_t)i) : (uint32_t)kOrderBuckets;
        const uint32_t grp = __match_any_sync(0xFFFFFFFFu, b);
        if (i < n && lane == (uint32_t)__ffs(grp) - 1u) atomicAdd(&cnt[b], (uint32_t)__popc(grp));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t sum = 0;
        for (int b = 0; b < kOrderBuckets; ++b) { const uint32_t c = cnt[b]; cnt[b] = sum; sum += c; }
    }
    __syncthreads();
    for (uint64_t b0 = 0; b0 < n; b0 += blockDim.x) {
        const uint64_t i = b0 + threadIdx.x;
        const uint32_t b = i < n ? key((uint32_t)i) : (uint32_t)kOrderBuckets;
        const uint32_t grp = __match_any_sync(0xFFFFFFFFu, b);
        const uint32_t lead = (uint32_t)__ffs(grp) - 1u;
        uint32_t pos = 0;
        if (i < n && lane == lead) pos = atomicAdd(&cnt[b], (uint32_t)__popc(grp));
        pos = __shfl_sync(0xFFFFFFFFu, pos, lead);
        if (i < n) perm[pos + (uint32_t)__popc(grp & ((1u << lane) - 1u))] = (uint32_t)i;
    }
}

// top of the score buckets: 32 candidates on the root router at slice 0
static int host_score_top(int n, int T) {
    const double x = 32.0 * (double)T * (double)(1u << n);
    unsigned long long bits;
    static_assert(sizeof(bits) == sizeof(x), "64-bit double");
    memcpy(&bits, &x, sizeof(bits));
    return (int)(bits >> 50);
}

static int score_grid(uint32_t n) {
    return (int)std::min<uint64_t>(((uint64_t)n + 7) / 8, 148ull * 16);
}

cudaError_t launch_order(const Params &p, uint32_t ntraj, uint32_t *perm, float *score, cudaStream_t s) {
    score_kernel<<<score_grid(ntraj), 256, 0, s>>>(p, ntraj, score);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ScoreKey key;
    key.score = score;
    key.ktop = host_score_top(p.n, p.T);
    order_kernel<ScoreKey><<<1, 1024, 0, s>>>(key, ntraj, perm);
    return cudaGetLastError();
}

cudaError_t launch_order_multi(const MultiParams &mp, int nmax, int tmax, uint32_t *perm, float *score,
                               cudaStream_t s) {
    const uint32_t n = mp.start[mp.nprob];
    score_kernel_multi<<<score_grid(n), 256, 0, s>>>(mp, score);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ScoreKey key;
    key.score = score;
    key.ktop = host_score_top(nmax, tmax);
    order_kernel<ScoreKey><<<1, 1024, 0, s>>>(key, n, perm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dump: Walsh-Hadamard transform of each (column, configuration) group at the
// second wall, plus the predicted good branches; normalised by sqrt(W).
__global__ void dump_finalize_kernel(const Params P, uint32_t n_in, uint32_t *out_n, uint32_t cap,
                                     uint32_t *o_addr, uint32_t *o_bus, uint64_t *o_hash, double *o_re,
                                     double *o_im) {
    const DumpOut &d = P.dump;
    const double W = d.scal[0];
    const double inv = W > 0 ? 1.0 / sqrt(W) : 0.0;
    const bool qubit = P.enc == QRAM_QUBIT;
    const uint32_t nw = qubit ? (1u << P.k) : 1u;
    const double hs = qubit ? sqrt(ldexp(1.0, -P.k)) : 1.0;
    // explicit groups: leader = first entry with the same (col, hash)
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_in; r += gridDim.x * blockDim.x) {
        bool leader = true;
        for (uint32_t q = 0; q < r; ++q)
            if (d.col[q] == d.col[r] && d.hash[q] == d.hash[r]) { leader = false; break; }
        if (!leader) continue;
        for (uint32_t w = 0; w < nw; ++w) {
            double re = 0.0, im = 0.0;
            for (uint32_t q = r; q < n_in; ++q) {
                if (d.col[q] != d.col[r] || d.hash[q] != d.hash[r]) continue;
                if (qubit) {
                    const double sg = (__popc(d.bus[q] & w) & 1u) ? -hs : hs;
                    re += sg * d.re[q]; im += sg * d.im[q];
                } else if (w == 0) { re += d.re[q]; im += d.im[q]; }
            }
            const uint32_t busw = qubit ? w : d.bus[r];
            const uint32_t o = atomicAdd(out_n, 1u);
            if (o < cap) {
                o_addr[o] = __ldg(P.addr + d.col[r]); o_bus[o] = busw; o_hash[o] = d.hash[r];
                o_re[o] = re * inv; o_im[o] = im * inv;
            }
        }
    }
    // branches in closed form (pruned mode, no jump fired): the good ones of
    // the eager form, or every branch of the lazy form
    if (P.mode != kPruned || d.scal[1] != 0.0 || d.scal[2] != 0.0) return;
    const bool all_closed = d.scal[3] != 0.0;
    const double g = P.gamma[0];
    const double a = sqrt(1.0 - g);
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < (uint32_t)P.D; b += gridDim.x * blockDim.x) {
        const uint32_t i = __ldg(P.addr + b);
        // eager form: the reference and the bad branches were explicit
        if (!all_closed) {
            if (P.o_badbits && ((P.o_badbits[i >> 5] >> (i & 31u)) & 1u)) continue;
            if ((int)b == *P.o_ref) continue;
        }
        int E = 0;
        const int n = P.n, T = P.T;
        for (int l = 0; l < n; ++l)
            if (!qubit || routed_bit(i, n, l)) E += T - 4 * l - 2;
        const uint32_t j = __ldg(P.bus + b), dm = __ldg(P.mem + i);
        if (!qubit) for (int t = 0; t < P.k; ++t) E += n * ((int)((j >> t) & 1u) + (int)(((j ^ dm) >> t) & 1u));
        double ae = 1.0;
        for (int q = 0; q < E; ++q) ae *= a;
        const double re0 = __ldg(P.amp_re + b), im0 = __ldg(P.amp_im + b);
        if (qubit) {
            double an = 1.0;
            for (int q = 0; q < 2 * n; ++q) an *= a;
            const double al = 0.5 * (1.0 + an), be = 0.5 * (1.0 - an);
            const uint32_t bout = j ^ dm;
            for (uint32_t w = 0; w < nw; ++w) {
                const int hw = __popc(w ^ bout);
                if (P.dump_wmax >= 0 && hw > P.dump_wmax) continue;        // low-weight truncation
                double A = ae;
                for (int q = 0; q < P.k; ++q) A *= q < hw ? be : al;
                const uint32_t o = atomicAdd(out_n, 1u);
                if (o < cap) { o_addr[o] = i; o_bus[o] = w; o_hash[o] = 0; o_re[o] = re0 * A * inv; o_im[o] = im0 * A * inv; }
            }
        } else {
            const uint32_t o = atomicAdd(out_n, 1u);
            if (o < cap) { o_addr[o] = i; o_bus[o] = j ^ dm; o_hash[o] = 0; o_re[o] = re0 * ae * inv; o_im[o] = im0 * ae * inv; }
        }
    }
}

cudaError_t launch_dump_finalize(const Params &p, uint32_t n_in, uint32_t *out_n, uint32_t cap,
                                 uint32_t *o_addr, uint32_t *o_bus, uint64_t *o_hash, double *o_re,
                                 double *o_im, cudaStream_t s) {
    dump_finalize_kernel<<<8, 128, 0, s>>>(p, n_in, out_n, cap, o_addr, o_bus, o_hash, o_re, o_im);
    return cudaGetLastError();
}

}  // namespace qram
