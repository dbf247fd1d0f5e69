/*
 * qram_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * trajectory simulation of amplitude-damped bucket-brigade QRAM.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (paper section / equation cited at each step):
 *   - the (n,k)-QRAM query of Eq. (1) run through the time-sliced bucket
 *     brigade schedule of Sec. II.A (T = 6n + 2k slices, Eqs. (2)-(4));
 *   - after the gates of every slice 1..T-1, one joint damping layer on all
 *     M = 2(2^n - 1) tree sites (Sec. II.B, Eqs. (5)-(6)), resolved by the
 *     joint sampler of Sec. IV.D (Eqs. (17)-(21)): candidate set drawn in
 *     advance, one auxiliary draw over the mask weights, K_J applied to the
 *     coherent state, normalisation once per layer;
 *   - a full evolution of EVERY input branch: the state is the unnormalised
 *     sparse dictionary {(i, j, Q) -> c} of App. A, Eq. (27), and every gate
 *     acts entry by entry;
 *   - the bad-address union R of Algorithm 1 (subtree rule Eq. (7) for the
 *     qutrit encoding, family-divergence rule Eq. (9) for the qubit
 *     encoding), reported beside the evolution (the full evolution does not
 *     use it);
 *   - the final tree measurement and the per-trajectory fidelity.
 *
 * Readings of the paper that this file fixes (where the paper is silent):
 *   S1 schedule: address bit l (the bit routed at tree layer l, i.e. address
 *      bit n-1-l, most significant bit at the root) is copied into d_0 at
 *      slice 2l+1, descends one layer per slice through the controlled swaps
 *      of layers 0..l-1 at slices 2l+1+m (m = 1..l), is swapped into the
 *      router of layer l at slice 3l+2, and leaves along the mirror image
 *      (slice s -> T - s).  Data qubit t enters d_0 at 2n+2t+1 (Eq. (3)),
 *      descends through layers 0..n-2 at 2n+2t+1+m, is fetched at the leaf
 *      layer at 3n+2t+1, climbs at 3n+2t+1+m and leaves at 4n+2t+1.  This
 *      reading reproduces the damping rows of Tab. IV exactly.
 *   S2 qubit encoding (App. C): copy-in/out = CNOT from the address bit into
 *      d_0; bus swaps are SWAPs; a controlled swap of layer L acts on every
 *      node of L (router 0 -> left child, 1 -> right child); the fetch is a
 *      phase -1 on a leaf data slot holding 1 when bit t of the routed cell
 *      is set; Hadamard walls on the bus before the gates of slice 2n+1 and
 *      after the gates of slice 4n+2k-1.
 *   S3 qutrit encoding: address bit 0 -> L, 1 -> R; data bit 0 -> W,
 *      1 -> R; copy-in/out is the permutation W<->L (bit 0) or W<->R (bit 1)
 *      on d_0; a router at W swaps nothing; a bus swap exchanges a qubit
 *      0/1 with W/R and leaves a slot holding L alone; the fetch is W<->R on
 *      the leaf data slot of a node whose router is L/R when the routed
 *      memory bit is 1.
 *   S4 random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *      counter = (c0, c1 | stream << 24, traj_lo, traj_hi) with streams
 *      FAULT=1, AUX=2, FINAL=3.  AUX/FINAL: c0 = 0, c1 = slice (0 for FINAL),
 *      u = (w >> 11) * 2^-53 with w = word0 | word1 << 32.
 *      FAULT: every (slice, site) pair is a candidate independently with
 *      probability gamma.  The pairs are numbered x = (slice - 1) * M + site
 *      (M = 2 * nodes) and cut into blocks of 2048; inside block g the
 *      candidates follow from geometric gaps.  Draw r of block g is the
 *      64-bit word (0,1) (r even) or (2,3) (r odd) of the counter
 *      (g, r / 2, ...).  With thr = floor(gamma * 2^64), q_0 = 2^64 - thr
 *      and q_{m+1} = floor(q_m^2 / 2^64) (64-bit fixed-point powers of
 *      1 - gamma), the gap of a word u is built greedily from m = 12 down
 *      to 0: starting from acc = 2^64 - 1, j gains 2^m whenever
 *      floor(acc * q_m / 2^64) > u (and acc takes that value); so
 *      P(gap >= j) = (1 - gamma)^j up to 64-bit rounding.  A gap that
 *      reaches the block end ends the block.  gamma with thr = 0 draws none.
 *   S4b depolarizing faults (Sec. II.B; App. A): every (slice, site) pair
 *      carries a fault with probability eps, drawn like the FAULT stream but
 *      on stream PAULI=4; the operator of the event found by draw r of block
 *      g is floor(word0 * ntypes / 2^32) of counter (g, r | 5 << 24, ...):
 *      qubits Z, X, XZ (ntypes 3), qutrits the eight Weyl operators X^a Z^b
 *      in row order of (a, b) (ntypes 8).  Events act after the gates (and
 *      the walls) of their slice and before its damping layer, and mark
 *      bad(v) like damping candidates.  Reading: every tree site is active
 *      in every slice (App. C's "routing front" is not defined in the
 *      paper); parity unpinned against Tab. IV's Pauli row, pinned against
 *      the density-matrix oracle under the same reading.
 *   S5 canonical mask order: the empty mask first, then masks as sorted
 *      lists of (site, level) compared lexicographically, a proper prefix
 *      first; the selected J is the first mask whose cumulative weight
 *      exceeds u * W.  The final tree configuration Q is drawn the same way
 *      over configurations (ground first).
 *   S6 fidelity: F = |<psi_id, 0_tree | psi>|^2 / <psi_Q|psi_Q> when the
 *      sampled Q is the ground configuration, else 0; its trajectory mean is
 *      the density-matrix fidelity of App. C.
 *   S7 channel: amplitude damping (Eqs. (5)-(6)) by default.  The outlook
 *      (Sec. VII) names dephasing as a further channel with a diagonal
 *      no-jump operator; it is taken here as the phase-damping channel with
 *      the same no-jump operator K0 = diag(1, a) (qutrit diag(1, a, a)) and
 *      the jump K1 = sqrt(gamma)|1><1| (qutrit sqrt(gamma)|L><L|,
 *      sqrt(gamma)|R><R|), so that K_J^dagger K_J is the same diagonal as
 *      for damping and the joint sampler of Sec. IV.D applies unchanged
 *      (Theorem 3's argument only uses that diagonal); a jump projects onto
 *      the components holding the site excited instead of lowering it.
 *      Heating (the outlook's qutrit heating channel; also run for qubits)
 *      is taken as the diagonal no-jump operator K0 = diag(a, 1, 1) on
 *      {W, L, R} (qubit diag(a, 1)) with the jumps sqrt(gamma/2)|L><W| and
 *      sqrt(gamma/2)|R><W| (qubit sqrt(gamma)|1><0|).  K_J^dagger K_J is again
 *      diagonal, so the joint sampler applies with the masks taken over the
 *      ground sites: J = {(q, level_q) : q in C, x_q = W}, each candidate's
 *      target level (qutrit) drawn with the candidates: bit 0 of word 0 of
 *      counter (site, slice | 6 << 24, traj) on stream HEAT=6 (0 -> L,
 *      1 -> R).  K0 then weighs a component by a per ground site outside J,
 *      i.e. by a^(-#excited) relative to a factor common to all.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define OR_MAXE 64          /* max excited sites per component */
#define OR_MAXG 64          /* max gates per slice */

enum { OR_OK = 0, OR_E_ARG = 1, OR_E_OOM = 2, OR_E_SCHED = 3, OR_E_CAP = 4 };
enum { G_LOAD = 1, G_UNLOAD, G_BUS, G_ISWAP, G_CSWAP, G_FETCH };
enum { ENC_QUTRIT = 0, ENC_QUBIT = 1 };
enum { LV_W = 0, LV_L = 1, LV_R = 2 };   /* qubit: 0 / 1 use LV_W / LV_L */
enum { CH_DAMPING = 0, CH_DEPHASING = 1, CH_HEATING = 2 };  /* the per-slice channel (S7) */

typedef struct {
    int32_t encoding, n, k;
    const uint8_t *memory;            /* 2^n cells, bit t = d_i^(t) */
    int32_t D;
    const uint32_t *addr, *bus;       /* D input columns */
    const double *amp_re, *amp_im;
} oproblem;

/* optional fixed history for one trajectory (tests; Sec. VI.A "fixed noise
 * histories").  Arrays may be NULL. */
typedef struct {
    int32_t ncand;
    const int32_t *cand_slice, *cand_site;   /* replaces the FAULT draws */
    const double *aux_u;                     /* [T] ; NaN = use the AUX stream */
    double final_u;                          /* NaN = use the FINAL stream */
    int32_t nflip;
    const int32_t *flip_slice, *flip_site;   /* X flips after the gates (qubit) */
    double eps;                              /* depolarizing strength (sampled events) */
    int32_t stop_slice;                      /* > 0: stop after this slice's damping layer and
                                              * return that state (an observation point for tests;
                                              * the outputs then describe the partial query) */
    int32_t channel;                         /* CH_DAMPING (0), CH_DEPHASING (1) or CH_HEATING (2), S7 */
} ohist;

typedef struct {
    double fidelity, fidelity_unsampled, p_ground;
    uint32_t ncand, bad;
    int32_t ref;
    uint32_t jumps, first_jump_slice, jump_sites;
    uint32_t q_ground, status;
} otraj_out;

typedef struct {
    uint32_t addr, bus;
    int32_t ne;
    uint32_t site[OR_MAXE];
    uint8_t lvl[OR_MAXE];
    double re, im;
} ocomp;

typedef struct { ocomp *c; size_t n, cap; } ostate;

typedef struct { int kind, p; } ogate;
typedef struct {
    int n, k, T, M;
    int ng[1024];
    ogate g[1024][OR_MAXG];
} osched;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the published definition (Salmon et al. 2011) */
static void philox(const uint32_t ctr_in[4], uint64_t seed, uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t node, uint32_t slice, uint32_t stream,
                 uint64_t traj, uint32_t out[4])
{
    uint32_t ctr[4] = { node, slice | (stream << 24), (uint32_t)traj, (uint32_t)(traj >> 32) };
    philox(ctr, seed, out);
}

static double uniform53(uint32_t w0, uint32_t w1)
{
    uint64_t w = (uint64_t)w0 | ((uint64_t)w1 << 32);
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t oracle_threshold(double gamma) { return (uint64_t)ldexp(gamma, 64); }

void oracle_philox(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) { philox(ctr, seed, out); }

/* ------------------------------------------------------------------------ */
/* schedule (Sec. II.A, Eqs. (2)-(4); App. C gate list)                     */

static int layer_of(uint32_t v) { int l = 0; while ((2u << l) - 1 <= v) l++; return l; }

static void add_gate(osched *S, int s, int kind, int p)
{
    for (int i = 0; i < S->ng[s]; i++)
        if (S->g[s][i].kind == kind && S->g[s][i].p == p) return;   /* one gate */
    S->g[s][S->ng[s]].kind = kind;
    S->g[s][S->ng[s]].p = p;
    S->ng[s]++;
}

/* slots a gate touches (read or write): tree sites 0..M-1, address bits
 * M..M+n-1, bus qubits M+n..M+n+k-1 */
static int mark_slots(const osched *S, ogate g, uint8_t *used)
{
    int M = S->M, n = S->n;
#define USE(x) do { if (used[(x)]) return 1; used[(x)] = 1; } while (0)
    switch (g.kind) {
    case G_LOAD: case G_UNLOAD: USE(1); USE(M + g.p); break;
    case G_BUS: USE(1); USE(M + n + g.p); break;
    case G_ISWAP:
        for (uint32_t v = (1u << g.p) - 1; v < (2u << g.p) - 1; v++) { USE(2 * v); USE(2 * v + 1); }
        break;
    case G_CSWAP:
        for (uint32_t v = (1u << g.p) - 1; v < (2u << g.p) - 1; v++) {
            USE(2 * v); USE(2 * v + 1); USE(2 * (2 * v + 1) + 1); USE(2 * (2 * v + 2) + 1);
        }
        break;
    case G_FETCH:
        for (uint32_t v = (1u << (n - 1)) - 1; v < (1u << n) - 1; v++) { USE(2 * v); USE(2 * v + 1); }
        break;
    }
#undef USE
    return 0;
}

static int build_schedule(int n, int k, osched *S)
{
    if (n < 1 || k < 1 || k > n || 6 * n + 2 * k >= 1024) return OR_E_ARG;
    memset(S->ng, 0, sizeof(S->ng));
    S->n = n; S->k = k; S->T = 6 * n + 2 * k; S->M = 2 * ((1 << n) - 1);
    int T = S->T;
    for (int l = 0; l < n; l++) {                 /* address bit routed at layer l */
        add_gate(S, 2 * l + 1, G_LOAD, l);
        for (int m = 1; m <= l; m++) add_gate(S, 2 * l + 1 + m, G_CSWAP, m - 1);
        add_gate(S, 3 * l + 2, G_ISWAP, l);
        add_gate(S, T - 3 * l - 2, G_ISWAP, l);
        for (int m = 1; m <= l; m++) add_gate(S, T - 2 * l - 1 - m, G_CSWAP, m - 1);
        add_gate(S, T - 2 * l - 1, G_UNLOAD, l);
    }
    for (int t = 0; t < k; t++) {                 /* data qubit t, Eq. (3) */
        add_gate(S, 2 * n + 2 * t + 1, G_BUS, t);
        for (int m = 1; m <= n - 1; m++) add_gate(S, 2 * n + 2 * t + 1 + m, G_CSWAP, m - 1);
        add_gate(S, 3 * n + 2 * t + 1, G_FETCH, t);
        for (int m = 1; m <= n - 1; m++) add_gate(S, 3 * n + 2 * t + 1 + m, G_CSWAP, n - 1 - m);
        add_gate(S, 4 * n + 2 * t + 1, G_BUS, t);
    }
    /* every slice's gates must act on disjoint slots */
    uint8_t *used = malloc((size_t)S->M + n + k);
    if (!used) return OR_E_OOM;
    for (int s = 1; s < T; s++) {
        memset(used, 0, (size_t)S->M + n + k);
        for (int i = 0; i < S->ng[s]; i++)
            if (mark_slots(S, S->g[s][i], used)) { free(used); return OR_E_SCHED; }
    }
    free(used);
    return OR_OK;
}

int oracle_schedule(int n, int k, int32_t *out_kind, int32_t *out_param, int32_t *out_slice, int cap, int *count)
{
    osched *S = malloc(sizeof(osched));
    if (!S) return OR_E_OOM;
    int rc = build_schedule(n, k, S);
    if (rc) { free(S); return rc; }
    int c = 0;
    for (int s = 1; s < S->T; s++)
        for (int i = 0; i < S->ng[s]; i++) {
            if (c < cap) { out_kind[c] = S->g[s][i].kind; out_param[c] = S->g[s][i].p; out_slice[c] = s; }
            c++;
        }
    *count = c;
    free(S);
    return c > cap ? OR_E_CAP : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* component helpers: the tree configuration Q is the sorted list of sites  */
/* that are not in the ground level (|0> or |W>), with their level.         */

static int get_lvl(const ocomp *x, uint32_t site)
{
    for (int i = 0; i < x->ne; i++) if (x->site[i] == site) return x->lvl[i];
    return LV_W;
}

static int sort_comp(ocomp *x)
{
    for (int i = 1; i < x->ne; i++) {             /* insertion sort by site */
        uint32_t s = x->site[i]; uint8_t l = x->lvl[i]; int j = i - 1;
        while (j >= 0 && x->site[j] > s) { x->site[j + 1] = x->site[j]; x->lvl[j + 1] = x->lvl[j]; j--; }
        x->site[j + 1] = s; x->lvl[j + 1] = l;
    }
    return 0;
}

static int set_lvl(ocomp *x, uint32_t site, int lvl)
{
    for (int i = 0; i < x->ne; i++)
        if (x->site[i] == site) {
            if (lvl == LV_W) { x->site[i] = x->site[x->ne - 1]; x->lvl[i] = x->lvl[x->ne - 1]; x->ne--; sort_comp(x); }
            else x->lvl[i] = (uint8_t)lvl;
            return 0;
        }
    if (lvl == LV_W) return 0;
    if (x->ne >= OR_MAXE) return OR_E_CAP;
    x->site[x->ne] = site; x->lvl[x->ne] = (uint8_t)lvl; x->ne++;
    sort_comp(x);
    return 0;
}

static int push(ostate *st, const ocomp *x)
{
    if (st->n == st->cap) {
        size_t nc = st->cap ? 2 * st->cap : 64;
        ocomp *p = realloc(st->c, nc * sizeof(ocomp));
        if (!p) return OR_E_OOM;
        st->c = p; st->cap = nc;
    }
    st->c[st->n++] = *x;
    return 0;
}

/* key order: address, bus word, tree configuration */
static int cmp_config(const ocomp *a, const ocomp *b)
{
    int m = a->ne < b->ne ? a->ne : b->ne;
    for (int i = 0; i < m; i++) {
        if (a->site[i] != b->site[i]) return a->site[i] < b->site[i] ? -1 : 1;
        if (a->lvl[i] != b->lvl[i]) return a->lvl[i] < b->lvl[i] ? -1 : 1;
    }
    return a->ne < b->ne ? -1 : (a->ne > b->ne ? 1 : 0);
}
static int cmp_key(const void *pa, const void *pb)
{
    const ocomp *a = pa, *b = pb;
    if (a->addr != b->addr) return a->addr < b->addr ? -1 : 1;
    if (a->bus != b->bus) return a->bus < b->bus ? -1 : 1;
    return cmp_config(a, b);
}

/* sort by key and add the amplitudes of equal keys; drop exact zeros */
static void merge_equal(ostate *st)
{
    qsort(st->c, st->n, sizeof(ocomp), cmp_key);
    size_t w = 0;
    for (size_t r = 0; r < st->n; r++) {
        if (w > 0 && cmp_key(&st->c[w - 1], &st->c[r]) == 0) {
            st->c[w - 1].re += st->c[r].re; st->c[w - 1].im += st->c[r].im;
        } else st->c[w++] = st->c[r];
    }
    size_t z = 0;
    for (size_t r = 0; r < w; r++)
        if (st->c[r].re != 0.0 || st->c[r].im != 0.0) st->c[z++] = st->c[r];
    st->n = z;
}

/* Hadamard on every bus qubit (App. C "Hadamard walls on the bus") */
static int hadamard_wall(ostate *st, int k)
{
    ostate out = { 0 };
    double s = pow(2.0, -0.5 * k);
    for (size_t r = 0; r < st->n; r++) {
        ocomp x = st->c[r];
        for (uint32_t c = 0; c < (1u << k); c++) {
            ocomp y = x;
            int par = __builtin_popcount(x.bus & c) & 1;
            y.bus = c;
            y.re = (par ? -s : s) * x.re;
            y.im = (par ? -s : s) * x.im;
            if (push(&out, &y)) { free(out.c); return OR_E_OOM; }
        }
    }
    free(st->c);
    *st = out;
    merge_equal(st);
    return 0;
}

/* apply one gate to one component (entry by entry, App. A) */
static int apply_gate(const osched *S, const oproblem *P, ogate g, ocomp *x)
{
    int n = S->n, qubit = P->encoding == ENC_QUBIT;
    switch (g.kind) {
    case G_LOAD: case G_UNLOAD: {
        int b = (x->addr >> (n - 1 - g.p)) & 1;      /* address bit routed at layer p */
        int d0 = get_lvl(x, 1);
        int nd;
        if (qubit) nd = d0 ^ b;                       /* CNOT into d_0 */
        else {
            int tgt = b ? LV_R : LV_L;               /* W <-> L or W <-> R */
            nd = d0 == LV_W ? tgt : (d0 == tgt ? LV_W : d0);
        }
        return set_lvl(x, 1, nd);
    }
    case G_BUS: {
        int d0 = get_lvl(x, 1);
        int b = (x->bus >> g.p) & 1;
        if (qubit) {
            x->bus = (x->bus & ~(1u << g.p)) | ((uint32_t)(d0 & 1) << g.p);
            return set_lvl(x, 1, b);
        }
        if (d0 == LV_L) return 0;                     /* L untouched */
        x->bus = (x->bus & ~(1u << g.p)) | ((uint32_t)(d0 == LV_R) << g.p);
        return set_lvl(x, 1, b ? LV_R : LV_W);
    }
    case G_ISWAP: {
        /* swap a_v <-> d_v for every node v of layer p: map each excited site */
        uint32_t lo = (1u << g.p) - 1, hi = (2u << g.p) - 1;
        for (int i = 0; i < x->ne; i++) {
            uint32_t v = x->site[i] >> 1;
            if (v >= lo && v < hi) x->site[i] ^= 1u;
        }
        return sort_comp(x);
    }
    case G_CSWAP: {
        /* for every node v of layer p: swap d_v with d of the child its router
         * selects (qubit: 0 -> left, 1 -> right; qutrit: W -> none).  The
         * routers are read before the swap and are not moved by it. */
        uint32_t lo = (1u << g.p) - 1, hi = (2u << g.p) - 1;
        uint32_t newsite[OR_MAXE];
        for (int i = 0; i < x->ne; i++) {
            uint32_t q = x->site[i], v = q >> 1;
            newsite[i] = q;
            if ((q & 1u) == 0) continue;                       /* routers do not move */
            if (v >= lo && v < hi) {                           /* parent side */
                int r = get_lvl(x, 2 * v);
                if (!qubit && r == LV_W) continue;
                uint32_t child = qubit ? 2 * v + 1 + (uint32_t)r : 2 * v + (uint32_t)r;
                newsite[i] = 2 * child + 1;
            } else if (v >= hi && v < 2 * hi + 1) {            /* child side, layer p+1 */
                uint32_t par = (v - 1) / 2;
                int r = get_lvl(x, 2 * par);
                if (!qubit && r == LV_W) continue;
                uint32_t child = qubit ? 2 * par + 1 + (uint32_t)r : 2 * par + (uint32_t)r;
                if (child == v) newsite[i] = 2 * par + 1;
            }
        }
        for (int i = 0; i < x->ne; i++) x->site[i] = newsite[i];
        return sort_comp(x);
    }
    case G_FETCH: {
        uint32_t lo = (1u << (n - 1)) - 1, hi = (1u << n) - 1;
        if (qubit) {
            /* Z on d_v controlled by the routed cell's bit t (phase kickback) */
            for (int i = 0; i < x->ne; i++) {
                uint32_t q = x->site[i], v = q >> 1;
                if ((q & 1u) == 0 || v < lo || v >= hi) continue;
                uint32_t cell = 2 * (v - lo) + (uint32_t)get_lvl(x, 2 * v);
                if ((P->memory[cell] >> g.p) & 1) { x->re = -x->re; x->im = -x->im; }
            }
            return 0;
        }
        /* qutrit: W <-> R on d_v of every leaf node whose router is L or R */
        uint32_t flip[OR_MAXE]; int nf = 0;
        for (int i = 0; i < x->ne; i++) {
            uint32_t q = x->site[i], v = q >> 1;
            if ((q & 1u) != 0 || v < lo || v >= hi) continue;
            uint32_t cell = 2 * (v - lo) + (x->lvl[i] == LV_R ? 1u : 0u);
            if ((P->memory[cell] >> g.p) & 1) flip[nf++] = 2 * v + 1;
        }
        for (int i = 0; i < nf; i++) {
            int d = get_lvl(x, flip[i]);
            int nd = d == LV_W ? LV_R : (d == LV_R ? LV_W : d);
            int rc = set_lvl(x, flip[i], nd);
            if (rc) return rc;
        }
        return 0;
    }
    }
    return OR_E_ARG;
}

/* ------------------------------------------------------------------------ */
/* joint damping layer (Sec. IV.D)                                          */

typedef struct { int n; uint32_t site[OR_MAXE]; uint8_t lvl[OR_MAXE]; } omask;

static int cmp_mask(const omask *a, const omask *b)
{
    int m = a->n < b->n ? a->n : b->n;
    for (int i = 0; i < m; i++) {
        if (a->site[i] != b->site[i]) return a->site[i] < b->site[i] ? -1 : 1;
        if (a->lvl[i] != b->lvl[i]) return a->lvl[i] < b->lvl[i] ? -1 : 1;
    }
    return a->n < b->n ? -1 : (a->n > b->n ? 1 : 0);
}

typedef struct { omask m; double w; size_t idx; } omw;
static int cmp_omw(const void *pa, const void *pb)
{
    const omw *a = pa, *b = pb;
    int c = cmp_mask(&a->m, &b->m);
    if (c) return c;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/* heating (S7): the target level of candidate (slice, site) */
static int heat_level(uint64_t seed, uint64_t traj, int slice, int32_t site, int qubit)
{
    if (qubit) return LV_L;
    uint32_t o[4];
    draw(seed, (uint32_t)site, (uint32_t)slice, 6u, traj, o);
    return (o[0] & 1u) ? LV_R : LV_L;
}

/* heating mask: the candidate sites x holds at the ground level, with the
 * candidates' target levels (lv[j] for cand[j]) */
static void mask_of_heat(const ocomp *x, const int32_t *cand, const uint8_t *lv, int nc, omask *m)
{
    m->n = 0;
    for (int j = 0; j < nc; j++)
        if (get_lvl(x, (uint32_t)cand[j]) == LV_W) { m->site[m->n] = (uint32_t)cand[j]; m->lvl[m->n] = lv[j]; m->n++; }
}

/* mask J(x) = C intersect X(x) with the levels of x (Eq. (21)) */
static void mask_of(const ocomp *x, const int32_t *cand, int nc, omask *m)
{
    m->n = 0;
    int i = 0, j = 0;
    while (i < x->ne && j < nc) {
        if (x->site[i] == (uint32_t)cand[j]) { m->site[m->n] = x->site[i]; m->lvl[m->n] = x->lvl[i]; m->n++; i++; j++; }
        else if (x->site[i] < (uint32_t)cand[j]) i++;
        else j++;
    }
}

/* One joint layer on the state: candidate set cand[0..nc) (sorted),
 * auxiliary uniform u.  Selects J (written to Jout), applies K_J of Eq. (17)
 * and normalises.  Returns 0 on success. */
static int joint_layer(ostate *st, const int32_t *cand, const uint8_t *hlv, int nc, double gamma, double u,
                       int channel, omask *Jout)
{
    double a = sqrt(1.0 - gamma), sg = sqrt(gamma);
    Jout->n = 0;
    if (nc > 0) {
        omw *list = malloc((st->n + 1) * sizeof(omw));
        if (!list) return OR_E_OOM;
        size_t nl = 0;
        double W = 0.0, w_empty = 0.0;
        for (size_t r = 0; r < st->n; r++) {
            const ocomp *x = &st->c[r];
            double w = x->re * x->re + x->im * x->im;
            W += w;
            omask m;
            if (channel == CH_HEATING) mask_of_heat(x, cand, hlv, nc, &m);
            else mask_of(x, cand, nc, &m);
            if (m.n == 0) w_empty += w;
            else { list[nl].m = m; list[nl].w = w; list[nl].idx = r; nl++; }
        }
        qsort(list, nl, sizeof(omw), cmp_omw);
        double t = u * W, cum = w_empty;
        int chosen = 0;                    /* 0: the empty mask */
        size_t pick = 0;
        if (!(cum > t)) {
            size_t r = 0;
            while (r < nl) {
                size_t e = r;
                double wj = 0.0;
                while (e < nl && cmp_mask(&list[e].m, &list[r].m) == 0) { wj += list[e].w; e++; }
                cum += wj;
                if (wj > 0.0) { chosen = 1; pick = r; }
                if (cum > t && wj > 0.0) break;
                r = e;
            }
        }
        if (chosen) *Jout = list[pick].m;
        free(list);
    }
    /* apply K_J: the jump operator on the sites of J, K0 elsewhere.  Amplitude
     * damping (S7): K1 = sqrt(g)|0><1| (qutrit: K1, K2 = sqrt(g)|W><L|,
     * sqrt(g)|W><R|) lowers the site to the ground level.  Dephasing (S7):
     * K1 = sqrt(g)|1><1| (qutrit: sqrt(g)|L><L|, sqrt(g)|R><R|) keeps it.
     * Either way a component that does not hold every site of J at its
     * level is annihilated, and K0 = diag(1, a) (diag(1, a, a)) gives a
     * factor a per excited site outside J. */
    size_t w = 0;
    if (channel == CH_HEATING) {
        /* heating: K_J needs every site of J at the ground level and raises it
         * to its target level; K0 gives a per ground site outside J, i.e.
         * a^(M - #excited - |J|): a^(-#excited) up to a factor common to all */
        for (size_t r = 0; r < st->n; r++) {
            ocomp x = st->c[r];
            int alive = 1;
            for (int j = 0; j < Jout->n; j++)
                if (get_lvl(&x, Jout->site[j]) != LV_W) { alive = 0; break; }
            if (!alive) continue;
            double f = 1.0;
            for (int e = 0; e < x.ne; e++) f /= a;
            for (int j = 0; j < Jout->n; j++)
                if (set_lvl(&x, Jout->site[j], Jout->lvl[j])) return OR_E_CAP;
            x.re *= f; x.im *= f;
            st->c[w++] = x;
        }
        st->n = w;
    } else
    for (size_t r = 0; r < st->n; r++) {
        ocomp x = st->c[r];
        int alive = 1;
        for (int j = 0; j < Jout->n; j++)
            if (get_lvl(&x, Jout->site[j]) != Jout->lvl[j]) { alive = 0; break; }
        if (!alive) continue;
        double f = 1.0;
        for (int j = 0; j < Jout->n; j++) {
            f *= sg;
            if (channel == CH_DAMPING) set_lvl(&x, Jout->site[j], LV_W);
        }
        const int outside = channel == CH_DAMPING ? x.ne : x.ne - Jout->n;
        for (int e = 0; e < outside; e++) f *= a;   /* K0 on the excited sites outside J */
        x.re *= f; x.im *= f;
        st->c[w++] = x;
    }
    st->n = w;
    double nrm = 0.0;
    for (size_t r = 0; r < st->n; r++) nrm += st->c[r].re * st->c[r].re + st->c[r].im * st->c[r].im;
    if (nrm > 0.0) {
        double s = 1.0 / sqrt(nrm);
        for (size_t r = 0; r < st->n; r++) { st->c[r].re *= s; st->c[r].im *= s; }
    }
    return 0;
}

/* exported for the single-layer exactness test of Theorem 3 */
int oracle_joint_layer(int32_t ncomp, uint32_t *addr, uint32_t *bus, int32_t *ne, uint32_t *sites,
                       uint8_t *lvls, double *re, double *im, int32_t *ncomp_out,
                       const int32_t *cand, int32_t nc, double gamma, double u,
                       int32_t *jn, uint32_t *jsite, uint8_t *jlvl, int32_t channel, const uint8_t *hlv)
{
    if (channel != CH_DAMPING && channel != CH_DEPHASING && channel != CH_HEATING) return OR_E_ARG;
    if (channel == CH_HEATING && !hlv) return OR_E_ARG;
    ostate st = { 0 };
    for (int r = 0; r < ncomp; r++) {
        ocomp x; memset(&x, 0, sizeof(x));
        x.addr = addr[r]; x.bus = bus[r]; x.ne = ne[r]; x.re = re[r]; x.im = im[r];
        if (x.ne > OR_MAXE) { free(st.c); return OR_E_CAP; }
        for (int e = 0; e < x.ne; e++) { x.site[e] = sites[r * OR_MAXE + e]; x.lvl[e] = lvls[r * OR_MAXE + e]; }
        sort_comp(&x);
        if (push(&st, &x)) { free(st.c); return OR_E_OOM; }
    }
    omask J;
    int rc = joint_layer(&st, cand, hlv, nc, gamma, u, channel, &J);
    if (rc) { free(st.c); return rc; }
    *jn = J.n;
    for (int j = 0; j < J.n; j++) { jsite[j] = J.site[j]; jlvl[j] = J.lvl[j]; }
    *ncomp_out = (int32_t)st.n;
    for (size_t r = 0; r < st.n; r++) {
        addr[r] = st.c[r].addr; bus[r] = st.c[r].bus; ne[r] = st.c[r].ne; re[r] = st.c[r].re; im[r] = st.c[r].im;
        for (int e = 0; e < st.c[r].ne; e++) { sites[r * OR_MAXE + e] = st.c[r].site[e]; lvls[r * OR_MAXE + e] = st.c[r].lvl[e]; }
    }
    free(st.c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* classification (Eq. (7), Eq. (9), Algorithm 1 steps 1-2)                  */

/* leaf range [lo, hi) of node v (Eq. (7)) */
static void subtree_range(int n, uint32_t v, uint32_t *lo, uint32_t *hi)
{
    int l = layer_of(v);
    uint32_t p = v - ((1u << l) - 1);
    *lo = p << (n - l);
    *hi = (p + 1) << (n - l);
}

/* bad(v): qutrit -> subtree(v); qubit -> Eq. (9) */
void oracle_bad_range(int encoding, int n, uint32_t v, uint32_t *lo, uint32_t *hi)
{
    if (encoding == ENC_QUTRIT) { subtree_range(n, v, lo, hi); return; }
    if (v == 0) { *lo = 0; *hi = 1u << n; return; }
    uint32_t par = (v - 1) / 2;
    int right = (v % 2) == 0;
    if (right || par == 0) { subtree_range(n, v, lo, hi); return; }
    oracle_bad_range(encoding, n, par, lo, hi);
}

/* geometric gap of a 64-bit uniform word (S4) */
#define OR_GAP_BLOCK 2048u
#define OR_GAP_BITS 13
static uint64_t umulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }

static void gap_powers(uint64_t thr, uint64_t q[OR_GAP_BITS])
{
    q[0] = (uint64_t)0 - thr;                       /* 2^64 - thr, thr >= 1 */
    for (int m = 0; m + 1 < OR_GAP_BITS; m++) q[m + 1] = umulhi64(q[m], q[m]);
}

static uint32_t gap_of(uint64_t u, const uint64_t q[OR_GAP_BITS])
{
    uint64_t acc = ~(uint64_t)0;
    uint32_t j = 0;
    for (int m = OR_GAP_BITS - 1; m >= 0; m--) {
        uint64_t t = umulhi64(acc, q[m]);
        if (t > u) { acc = t; j += 1u << m; }
    }
    return j;
}

uint32_t oracle_gap(uint64_t u, double gamma)
{
    uint64_t q[OR_GAP_BITS];
    uint64_t thr = oracle_threshold(gamma);
    if (thr == 0) return 0xFFFFFFFFu;
    gap_powers(thr, q);
    return gap_of(u, q);
}

/* fault positions of one stream in (slice, site) order; with ct, also each
 * event's operator index (S4b); returns count */
static int sample_stream(const osched *S, uint64_t seed, uint64_t traj, double gamma, uint32_t stream,
                         uint32_t ntypes, int32_t **cs, int32_t **cq, int32_t **ct, int *nc_out);

static int sample_candidates(const osched *S, uint64_t seed, uint64_t traj, double gamma,
                             int32_t **cs, int32_t **cq, int *nc_out)
{
    return sample_stream(S, seed, traj, gamma, 1u, 0u, cs, cq, NULL, nc_out);
}

static int sample_stream(const osched *S, uint64_t seed, uint64_t traj, double gamma, uint32_t stream,
                         uint32_t ntypes, int32_t **cs, int32_t **cq, int32_t **ct, int *nc_out)
{
    uint64_t thr = oracle_threshold(gamma);
    int cap = 256, nc = 0;
    int32_t *a = malloc(cap * sizeof(int32_t)), *b = malloc(cap * sizeof(int32_t)), *c = malloc(cap * sizeof(int32_t));
    if (!a || !b || !c) { free(a); free(b); free(c); return OR_E_OOM; }
    *cs = a; *cq = b; *nc_out = 0;
    if (ct) *ct = c;
    if (thr == 0) { if (!ct) free(c); return 0; }
    uint64_t q[OR_GAP_BITS];
    gap_powers(thr, q);
    const uint64_t M = 2 * (((uint64_t)1 << S->n) - 1), X = (uint64_t)(S->T - 1) * M;
    for (uint64_t g = 0; g * OR_GAP_BLOCK < X; g++) {
        uint64_t pos = g * OR_GAP_BLOCK, end = pos + OR_GAP_BLOCK < X ? pos + OR_GAP_BLOCK : X;
        uint32_t o[4] = {0, 0, 0, 0};
        for (uint32_t r = 0;; r++) {
            if ((r & 1u) == 0) draw(seed, (uint32_t)g, r >> 1, stream, traj, o);
            uint64_t u = (r & 1u) ? ((uint64_t)o[2] | ((uint64_t)o[3] << 32)) : ((uint64_t)o[0] | ((uint64_t)o[1] << 32));
            uint32_t G = gap_of(u, q);
            if ((uint64_t)G >= end - pos) break;
            pos += G;
            if (nc == cap) {
                cap *= 2;
                int32_t *a2 = realloc(a, cap * sizeof(int32_t)), *b2 = realloc(b, cap * sizeof(int32_t));
                int32_t *c2 = realloc(c, cap * sizeof(int32_t));
                if (!a2 || !b2 || !c2) { free(a2 ? a2 : a); free(b2 ? b2 : b); free(c2 ? c2 : c); return OR_E_OOM; }
                a = a2; b = b2; c = c2;
            }
            a[nc] = (int32_t)(1 + pos / M); b[nc] = (int32_t)(pos % M);
            if (ntypes) {                               /* the event's operator: multiply-shift of a fresh word */
                uint32_t w[4];
                draw(seed, (uint32_t)g, r, 5u, traj, w);
                c[nc] = (int32_t)(((uint64_t)w[0] * ntypes) >> 32);
            }
            nc++;
            pos += 1;
        }
    }
    *cs = a; *cq = b; *nc_out = nc;
    if (ct) *ct = c; else free(c);
    return 0;
}

static void classify(const oproblem *P, int n, const int32_t *cq, int nc, uint8_t *badmap,
                     uint32_t *B, int32_t *ref)
{
    uint32_t N = 1u << n;
    memset(badmap, 0, N);
    for (int c = 0; c < nc; c++) {                  /* mark each fault, whatever its type */
        uint32_t lo, hi;
        oracle_bad_range(P->encoding, n, (uint32_t)cq[c] >> 1, &lo, &hi);
        for (uint32_t i = lo; i < hi; i++) badmap[i] = 1;
    }
    *B = 0; *ref = -1;
    for (int b = 0; b < P->D; b++) {
        if (badmap[P->addr[b]]) (*B)++;
        else if (*ref < 0) *ref = b;                /* first good branch */
    }
}

int oracle_sample_faults(const oproblem *P, uint64_t seed, uint64_t traj, double gamma,
                         int32_t *out_slice, int32_t *out_site, int32_t cap, int32_t *ncand,
                         uint8_t *badmap, uint32_t *B, int32_t *ref)
{
    osched *S = malloc(sizeof(osched));
    if (!S) return OR_E_OOM;
    int rc = build_schedule(P->n, P->k, S);
    if (rc) { free(S); return rc; }
    int32_t *cs, *cq; int nc;
    rc = sample_candidates(S, seed, traj, gamma, &cs, &cq, &nc);
    free(S);
    if (rc) return rc;
    for (int c = 0; c < nc && c < cap; c++) { out_slice[c] = cs[c]; out_site[c] = cq[c]; }
    *ncand = nc;
    classify(P, P->n, cq, nc, badmap, B, ref);
    free(cs); free(cq);
    return nc > cap ? OR_E_CAP : OR_OK;
}

/* depolarizing fault events of one trajectory (S4b): slice, site, operator */
int oracle_sample_paulis(const oproblem *P, uint64_t seed, uint64_t traj, double eps, int32_t *out_slice,
                         int32_t *out_site, int32_t *out_type, int32_t cap, int32_t *nev)
{
    osched *S = malloc(sizeof(osched));
    if (!S) return OR_E_OOM;
    int rc = build_schedule(P->n, P->k, S);
    if (rc) { free(S); return rc; }
    int32_t *ps, *pq, *pt; int np;
    rc = sample_stream(S, seed, traj, eps, 4u, P->encoding == ENC_QUBIT ? 3u : 8u, &ps, &pq, &pt, &np);
    free(S);
    if (rc) return rc;
    for (int e = 0; e < np && e < cap; e++) { out_slice[e] = ps[e]; out_site[e] = pq[e]; out_type[e] = pt[e]; }
    *nev = np;
    free(ps); free(pq); free(pt);
    return np > cap ? OR_E_CAP : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* one trajectory: full evolution of every branch                           */

static int check_problem(const oproblem *P)
{
    if (P->encoding != ENC_QUTRIT && P->encoding != ENC_QUBIT) return OR_E_ARG;
    if (P->n < 1 || P->n > 14 || P->k < 1 || P->k > P->n || P->k > 8) return OR_E_ARG;
    if (P->D < 1 || P->D > (1 << P->n)) return OR_E_ARG;
    return 0;
}

/* depolarizing fault (S4b): operator index t -> X^a Z^b with (a, b) the
 * (t+1)-th pair of {0..d-1}^2 in row order (qubit: Z, X, XZ; qutrit: the
 * eight Weyl operators), X|j> = |j+1 mod d>, Z|j> = w^j |j>, w = exp(2 pi i/d);
 * applied to one site of one component */
static int apply_weyl(ocomp *x, uint32_t site, int qubit, int t)
{
    const int d = qubit ? 2 : 3;
    const int a = (t + 1) / d, b = (t + 1) % d;
    const int j = get_lvl(x, site);                 /* qubit: LV_W = 0, LV_L = 1 */
    const int m = (b * j) % d;
    if (m) {                                        /* w^m: -1 (qubit); -1/2 +- i sqrt(3)/2 (qutrit) */
        const double c = qubit ? -1.0 : -0.5, sn = qubit ? 0.0 : (m == 1 ? 0.5 : -0.5) * sqrt(3.0);
        const double re = x->re * c - x->im * sn, im = x->re * sn + x->im * c;
        x->re = re; x->im = im;
    }
    return set_lvl(x, site, (j + a) % d);
}

static int run_traj(const oproblem *P, const osched *S, uint64_t seed, uint64_t traj, double gamma,
                    double eps, int channel, const ohist *H, otraj_out *out, ostate *dump, uint8_t *occupancy)
{
    int n = S->n, k = S->k, T = S->T, qubit = P->encoding == ENC_QUBIT;
    memset(out, 0, sizeof(*out));
    int32_t *cs = NULL, *cq = NULL; int nc = 0, rc;
    if (H && H->cand_slice) {
        nc = H->ncand;
        cs = malloc((nc + 1) * sizeof(int32_t)); cq = malloc((nc + 1) * sizeof(int32_t));
        if (!cs || !cq) { free(cs); free(cq); return OR_E_OOM; }
        for (int c = 0; c < nc; c++) { cs[c] = H->cand_slice[c]; cq[c] = H->cand_site[c]; }
        for (int i = 1; i < nc; i++) {                 /* order by (slice, site) */
            int32_t a = cs[i], b = cq[i]; int j = i - 1;
            while (j >= 0 && (cs[j] > a || (cs[j] == a && cq[j] > b))) { cs[j + 1] = cs[j]; cq[j + 1] = cq[j]; j--; }
            cs[j + 1] = a; cq[j + 1] = b;
        }
    } else if ((rc = sample_candidates(S, seed, traj, gamma, &cs, &cq, &nc))) return rc;
    out->ncand = (uint32_t)nc;
    /* depolarizing fault events (S4b) */
    int32_t *ps = NULL, *pq = NULL, *pt = NULL; int np = 0;
    if (eps > 0.0 && (rc = sample_stream(S, seed, traj, eps, 4u, qubit ? 3u : 8u, &ps, &pq, &pt, &np))) {
        free(cs); free(cq); return rc;
    }

    uint8_t *badmap = malloc(1u << n);
    int32_t *allq = malloc((size_t)(nc + np + 1) * sizeof(int32_t));
    if (!badmap || !allq) { free(badmap); free(allq); free(cs); free(cq); free(ps); free(pq); free(pt); return OR_E_OOM; }
    for (int c = 0; c < nc; c++) allq[c] = cq[c];
    for (int e = 0; e < np; e++) allq[nc + e] = pq[e];            /* every fault marks, whatever its type */
    classify(P, n, allq, nc + np, badmap, &out->bad, &out->ref);
    free(badmap); free(allq);

    /* initial sparse state: one component per input column, tree in ground */
    ostate st = { 0 };
    for (int b = 0; b < P->D; b++) {
        ocomp x; memset(&x, 0, sizeof(x));
        x.addr = P->addr[b]; x.bus = P->bus[b];
        x.re = P->amp_re[b]; x.im = P->amp_im[b];
        if ((rc = push(&st, &x))) goto fail;
    }

    for (int s = 1; s < T; s++) {
        if (qubit && s == 2 * n + 1) { if ((rc = hadamard_wall(&st, k))) goto fail; }
        for (int gi = 0; gi < S->ng[s]; gi++)
            for (size_t r = 0; r < st.n; r++)
                if ((rc = apply_gate(S, P, S->g[s][gi], &st.c[r]))) goto fail;
        if (qubit && s == 4 * n + 2 * k - 1) { if ((rc = hadamard_wall(&st, k))) goto fail; }
        if (H && H->flip_slice)                       /* injected X flips (qubit) */
            for (int f = 0; f < H->nflip; f++)
                if (H->flip_slice[f] == s)
                    for (size_t r = 0; r < st.n; r++) {
                        uint32_t q = (uint32_t)H->flip_site[f];
                        if ((rc = set_lvl(&st.c[r], q, get_lvl(&st.c[r], q) ? LV_W : LV_L))) goto fail;
                    }
        for (int e = 0; e < np; e++)                  /* depolarizing faults of this slice */
            if (ps[e] == s)
                for (size_t r = 0; r < st.n; r++)
                    if ((rc = apply_weyl(&st.c[r], (uint32_t)pq[e], qubit, pt[e]))) goto fail;
        if (occupancy)
            for (size_t r = 0; r < st.n; r++)
                for (int e = 0; e < st.c[r].ne; e++) occupancy[(size_t)s * S->M + st.c[r].site[e]] = 1;
        /* candidates of this slice, sorted by site */
        int c0 = 0; while (c0 < nc && cs[c0] < s) c0++;
        int c1 = c0; while (c1 < nc && cs[c1] == s) c1++;
        int32_t *cand = cq + c0; int ncs = c1 - c0;
        for (int i = 1; i < ncs; i++) { int32_t v = cand[i]; int j = i - 1; while (j >= 0 && cand[j] > v) { cand[j + 1] = cand[j]; j--; } cand[j + 1] = v; }
        double u = 0.0;
        if (ncs > 0) {
            if (H && H->aux_u && !isnan(H->aux_u[s])) u = H->aux_u[s];
            else { uint32_t o[4]; draw(seed, 0, (uint32_t)s, 2u, traj, o); u = uniform53(o[0], o[1]); }
        }
        omask J;
        uint8_t hlv[OR_MAXE * 64];
        if (channel == CH_HEATING) {
            if (ncs > (int)sizeof(hlv)) { rc = OR_E_CAP; goto fail; }
            for (int j = 0; j < ncs; j++) hlv[j] = (uint8_t)heat_level(seed, traj, s, cand[j], qubit);
        }
        if ((rc = joint_layer(&st, cand, hlv, ncs, gamma, u, channel, &J))) goto fail;
        if (J.n > 0) {
            if (out->jumps == 0) out->first_jump_slice = (uint32_t)s;
            out->jumps++;
            out->jump_sites += (uint32_t)J.n;
        }
        if (H && H->stop_slice == s) break;
    }

    /* final tree measurement (S5) and fidelity (S6) */
    {
        merge_equal(&st);
        /* sort by configuration (ground first) to walk configurations in order */
        double W = 0.0, Wg = 0.0, ore = 0.0, oim = 0.0;
        int32_t *col = malloc(sizeof(int32_t) << n);   /* address -> input column */
        if (!col) { rc = OR_E_OOM; goto fail; }
        for (uint32_t i = 0; i < (1u << n); i++) col[i] = -1;
        for (int b = 0; b < P->D; b++) col[P->addr[b]] = b;
        for (size_t r = 0; r < st.n; r++) {
            const ocomp *x = &st.c[r];
            double w = x->re * x->re + x->im * x->im;
            W += w;
            if (x->ne == 0) {
                Wg += w;
                int b = col[x->addr];                /* <psi_id| : c_b |i_b, j_b xor d_i> */
                if (b >= 0 && (P->bus[b] ^ (uint32_t)P->memory[x->addr]) == x->bus) {
                    ore += P->amp_re[b] * x->re + P->amp_im[b] * x->im;
                    oim += P->amp_re[b] * x->im - P->amp_im[b] * x->re;
                }
            }
        }
        free(col);
        double uf;
        if (H && !isnan(H->final_u)) uf = H->final_u;
        else { uint32_t o[4]; draw(seed, 0, 0, 3u, traj, o); uf = uniform53(o[0], o[1]); }
        /* canonical walk: ground configuration first; its weight decides */
        int ground = (Wg > uf * W) || (Wg > 0.0 && Wg >= W);
        double ov = ore * ore + oim * oim;
        out->p_ground = W > 0 ? Wg / W : 0.0;
        out->q_ground = (uint32_t)ground;
        out->fidelity = (ground && Wg > 0) ? ov / Wg : 0.0;
        out->fidelity_unsampled = W > 0 ? ov / W : 0.0;
    }
    if (dump) { *dump = st; st.c = NULL; }
    free(st.c); free(cs); free(cq); free(ps); free(pq); free(pt);
    return 0;
fail:
    free(st.c); free(cs); free(cq); free(ps); free(pq); free(pt);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* threaded ensemble driver                                                 */

typedef struct {
    const oproblem *P; const osched *S; uint64_t seed, traj0; int ntraj;
    const double *gamma; double eps; int channel; otraj_out *out; int next; int rc;
    pthread_mutex_t mu;
} ojob;

static void *worker(void *arg)
{
    ojob *J = arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int t = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (t >= J->ntraj) break;
        const double e = J->eps < 0.0 ? J->gamma[t] : J->eps;       /* eps < 0: eps = gamma */
        int rc = run_traj(J->P, J->S, J->seed, J->traj0 + (uint64_t)t, J->gamma[t], e, J->channel, NULL, &J->out[t],
                          NULL, NULL);
        if (rc) { pthread_mutex_lock(&J->mu); J->rc = rc; pthread_mutex_unlock(&J->mu); }
    }
    return NULL;
}

int oracle_run_ch(const oproblem *P, uint64_t seed, uint64_t traj0, int32_t ntraj, const double *gamma,
                  double eps, int32_t channel, int32_t nthreads, otraj_out *out);

int oracle_run(const oproblem *P, uint64_t seed, uint64_t traj0, int32_t ntraj,
               const double *gamma, int32_t nthreads, otraj_out *out)
{
    return oracle_run_ch(P, seed, traj0, ntraj, gamma, 0.0, CH_DAMPING, nthreads, out);
}

/* eps: depolarizing strength per (slice, site); eps < 0 takes eps = gamma
 * per trajectory (the paper's benchmark setting) */
int oracle_run_eps(const oproblem *P, uint64_t seed, uint64_t traj0, int32_t ntraj, const double *gamma,
                   double eps, int32_t nthreads, otraj_out *out)
{
    return oracle_run_ch(P, seed, traj0, ntraj, gamma, eps, CH_DAMPING, nthreads, out);
}

/* channel: CH_DAMPING, CH_DEPHASING or CH_HEATING (S7) */
int oracle_run_ch(const oproblem *P, uint64_t seed, uint64_t traj0, int32_t ntraj, const double *gamma,
                  double eps, int32_t channel, int32_t nthreads, otraj_out *out)
{
    if (channel != CH_DAMPING && channel != CH_DEPHASING && channel != CH_HEATING) return OR_E_ARG;
    int rc = check_problem(P);
    if (rc) return rc;
    osched *S = malloc(sizeof(osched));
    if (!S) return OR_E_OOM;
    if ((rc = build_schedule(P->n, P->k, S))) { free(S); return rc; }
    for (int t = 0; t < ntraj; t++) if (!(gamma[t] >= 0.0 && gamma[t] < 1.0)) { free(S); return OR_E_ARG; }
    ojob J;
    memset(&J, 0, sizeof(J));
    if (!(eps < 1.0)) { free(S); return OR_E_ARG; }
    J.P = P; J.S = S; J.seed = seed; J.traj0 = traj0; J.ntraj = ntraj; J.gamma = gamma; J.eps = eps; J.out = out;
    J.channel = channel;
    pthread_mutex_init(&J.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, worker, &J);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.mu);
    free(S);
    return J.rc;
}

/* one trajectory with an optional fixed history; optionally dumps the final
 * normalised state (sorted by address, bus word, configuration). */
int oracle_run_one(const oproblem *P, uint64_t seed, uint64_t traj, double gamma, const ohist *H,
                   otraj_out *out, int32_t cap, int32_t *ncomp, uint32_t *d_addr, uint32_t *d_bus,
                   int32_t *d_ne, uint32_t *d_sites, uint8_t *d_lvls, double *d_re, double *d_im)
{
    int rc = check_problem(P);
    if (rc) return rc;
    if (!(gamma >= 0.0 && gamma < 1.0)) return OR_E_ARG;
    osched *S = malloc(sizeof(osched));
    if (!S) return OR_E_OOM;
    if ((rc = build_schedule(P->n, P->k, S))) { free(S); return rc; }
    ostate st = { 0 };
    if (H && H->channel != CH_DAMPING && H->channel != CH_DEPHASING && H->channel != CH_HEATING) {
        free(S);
        return OR_E_ARG;
    }
    rc = run_traj(P, S, seed, traj, gamma, H ? H->eps : 0.0, H ? H->channel : CH_DAMPING, H, out, &st, NULL);
    free(S);
    if (rc) return rc;
    double W = 0.0;
    for (size_t r = 0; r < st.n; r++) W += st.c[r].re * st.c[r].re + st.c[r].im * st.c[r].im;
    double s = W > 0 ? 1.0 / sqrt(W) : 0.0;
    *ncomp = (int32_t)st.n;
    for (size_t r = 0; r < st.n && (int32_t)r < cap; r++) {
        d_addr[r] = st.c[r].addr; d_bus[r] = st.c[r].bus; d_ne[r] = st.c[r].ne;
        d_re[r] = st.c[r].re * s; d_im[r] = st.c[r].im * s;
        for (int e = 0; e < st.c[r].ne; e++) { d_sites[r * OR_MAXE + e] = st.c[r].site[e]; d_lvls[r * OR_MAXE + e] = st.c[r].lvl[e]; }
    }
    free(st.c);
    return (int32_t)st.n > cap ? OR_E_CAP : OR_OK;
}

/* noiseless occupancy: occ[s*M + site] = 1 when some component holds the
 * site excited after the gates of slice s (used for the vacuous-case count
 * of Sec. VI.B) */
int oracle_occupancy(const oproblem *P, uint8_t *occ)
{
    int rc = check_problem(P);
    if (rc) return rc;
    osched *S = malloc(sizeof(osched));
    if (!S) return OR_E_OOM;
    if ((rc = build_schedule(P->n, P->k, S))) { free(S); return rc; }
    memset(occ, 0, (size_t)S->T * S->M);
    ohist H; memset(&H, 0, sizeof(H));
    int32_t dummy = 0;
    H.cand_slice = &dummy; H.cand_site = &dummy; H.ncand = 0; H.final_u = 0.0;
    otraj_out o;
    rc = run_traj(P, S, 0, 0, 0.0, 0.0, CH_DAMPING, &H, &o, NULL, occ);
    free(S);
    return rc;
}

int oracle_maxe(void) { return OR_MAXE; }
