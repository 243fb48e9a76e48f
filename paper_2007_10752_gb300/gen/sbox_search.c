/*
 * sbox_search.c -- search for small circuits of 3-input lookup tables (the
 * sm_103a LOP3 instruction) that compute the four outputs of one DES S-box.
 *
 * Build-time tool of the code generator; it is not linked into the library.
 *
 * Every signal is a 64-bit truth table over the S-box's 6 inputs (bit x of
 * a table is the value at input x = b1..b6, b1 most significant).  A gate is
 * LUT(a, b, c) with an 8-bit table indexed by (a<<2 | b<<1 | c), which is
 * exactly the LOP3 immediate f(0xF0, 0xCC, 0xAA).
 *
 * Method (Kwan's multiplexer decomposition with gate reuse, adapted to
 * 3-input lookup tables): to realise a target table T on a care set M,
 *   1. reuse an existing gate equal to T (or to its complement) on M;
 *   2. else find one new LUT over any three existing gates that equals T on M;
 *   3. else find two new LUTs, LUT(a, b, LUT(c, d, e)), over existing gates;
 *   4. else split on an input variable v not yet used on this path:
 *      build A for T on M&~v, then B for T (or T^A) on M&v, and join them
 *      with one LUT(v, A, B); or, when T restricted to each value of a pair
 *      of inputs (v, w) is a function of one shared signal X, build X once
 *      and join with LUT(v, w, X).
 * Outputs are built one after another so later outputs reuse earlier gates.
 * Output complements are free (the consumer LOP3 absorbs them), so step 1
 * accepts either polarity and the caller records it.  Random restarts over
 * output orders and split variables keep the smallest circuit found.
 *
 * Usage: sbox_search T0 T1 T2 T3 iterations seed [lut2_limit [wide_depth [variant_depth
 *        [pair_tries]]]]
 *   T0..T3: hex truth tables of the four outputs (first output bit first).
 * Prints the best circuit: "gates N", then one line per gate
 * "g <id> <in0> <in1> <in2> <lut>" (ids 0..5 are the inputs b1..b6), then
 * "out <t> <gate> <neg>".
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXG 160
#define NIN 6

typedef struct {
    uint64_t tt;
    int16_t in[3];
    uint8_t lut;
} Gate;

typedef struct {
    Gate g[MAXG];
    int n;
    int out[4];
    uint8_t neg[4];
} Circ;

static uint64_t rng_state;
static uint64_t rnd(void) { /* xorshift64* */
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545F4914F6CDD1DULL;
}
static int rndn(int n) { return (int)(rnd() % (uint64_t)n); }

static int lut2_limit = 0; /* only try step 3 while the circuit has at most this many gates */
static int wide_depth = 1;     /* split nodes shallower than this try every variable */
static int variant_depth = 99; /* split nodes shallower than this try every join variant */

static inline uint64_t sel(uint64_t t, int bit) { return bit ? t : ~t; }

static uint64_t eval_lut(uint8_t lut, uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r = 0;
    for (int i = 0; i < 8; ++i)
        if ((lut >> i) & 1) r |= sel(a, i & 4) & sel(b, i & 2) & sel(c, i & 1);
    return r;
}

/* A LUT over (a, b, c) equal to T on M, if one exists. */
static int fit3(uint64_t a, uint64_t b, uint64_t c, uint64_t T, uint64_t M, uint8_t *lut) {
    uint8_t l = 0;
    for (int i = 0; i < 8; ++i) {
        uint64_t cls = M & sel(a, i & 4) & sel(b, i & 2) & sel(c, i & 1);
        uint64_t on = cls & T;
        if (on) {
            if (on != cls) return 0;
            l |= (uint8_t)(1u << i);
        }
    }
    *lut = l;
    return 1;
}

static int add_gate(Circ *C, int a, int b, int c, uint8_t lut) {
    if (C->n >= MAXG) return -1;
    Gate *g = &C->g[C->n];
    g->in[0] = (int16_t)a;
    g->in[1] = (int16_t)b;
    g->in[2] = (int16_t)c;
    g->lut = lut;
    g->tt = eval_lut(lut, C->g[a].tt, C->g[b].tt, C->g[c].tt);
    return C->n++;
}

static int find_existing(const Circ *C, uint64_t T, uint64_t M) {
    for (int i = 0; i < C->n; ++i) {
        uint64_t d = (C->g[i].tt ^ T) & M;
        if (d == 0 || d == M) return i;
    }
    return -1;
}

static int try_lut1(Circ *C, uint64_t T, uint64_t M) {
    int n = C->n;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            for (int k = j + 1; k < n; ++k) {
                uint8_t lut;
                if (fit3(C->g[i].tt, C->g[j].tt, C->g[k].tt, T, M, &lut))
                    return add_gate(C, i, j, k, lut);
            }
    return -1;
}

/* Step 3: T = LUT(a, b, h) with h = LUT(c, d, e).  For the pair (a, b) split
 * M into four classes q; where a class holds both zeros Z_q and ones O_q of
 * T, h must be one constant on Z_q and the other on O_q.  For a triple
 * (c, d, e), h is constant on each of its 8 classes p; solve for h(p) and
 * the per-class polarities by trying every polarity assignment. */
static int try_lut2(Circ *C, uint64_t T, uint64_t M) {
    int n = C->n;
    if (n > lut2_limit) return -1;
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            uint64_t Z[4], O[4];
            int mixed = 0, qs[4];
            for (int q = 0; q < 4; ++q) {
                uint64_t cls = M & sel(C->g[a].tt, q & 2) & sel(C->g[b].tt, q & 1);
                Z[q] = cls & ~T;
                O[q] = cls & T;
                if (Z[q] && O[q]) qs[mixed++] = q;
            }
            if (mixed == 0) continue; /* a 2-input LUT would have been found in step 2 */
            for (int c = 0; c < n; ++c)
                for (int d = c + 1; d < n; ++d)
                    for (int e = d + 1; e < n; ++e) {
                        /* per class p: which mixed q's zeros/ones it touches */
                        uint8_t touchZ[8], touchO[8];
                        int bad = 0;
                        for (int p = 0; p < 8 && !bad; ++p) {
                            uint64_t cls = sel(C->g[c].tt, p & 4) & sel(C->g[d].tt, p & 2) &
                                           sel(C->g[e].tt, p & 1);
                            touchZ[p] = touchO[p] = 0;
                            for (int m = 0; m < mixed; ++m) {
                                int q = qs[m];
                                int tz = (cls & Z[q]) != 0, to = (cls & O[q]) != 0;
                                if (tz && to) { bad = 1; break; }
                                touchZ[p] |= (uint8_t)(tz << m);
                                touchO[p] |= (uint8_t)(to << m);
                            }
                        }
                        if (bad) continue;
                        for (int alpha = 0; alpha < (1 << mixed); ++alpha) {
                            /* h(p) must be alpha_m where p touches Z of q_m, ~alpha_m on O */
                            uint8_t hl = 0;
                            int ok = 1;
                            for (int p = 0; p < 8 && ok; ++p) {
                                int need = -1;
                                for (int m = 0; m < mixed; ++m) {
                                    int am = (alpha >> m) & 1;
                                    if ((touchZ[p] >> m) & 1) {
                                        if (need >= 0 && need != am) { ok = 0; break; }
                                        need = am;
                                    }
                                    if ((touchO[p] >> m) & 1) {
                                        if (need >= 0 && need != !am) { ok = 0; break; }
                                        need = !am;
                                    }
                                }
                                if (need == 1) hl |= (uint8_t)(1u << p);
                            }
                            if (!ok) continue;
                            uint64_t h = eval_lut(hl, C->g[c].tt, C->g[d].tt, C->g[e].tt);
                            uint8_t top;
                            if (!fit3(C->g[a].tt, C->g[b].tt, h, T, M, &top)) continue;
                            int hid = add_gate(C, c, d, e, hl);
                            if (hid < 0) return -1;
                            return add_gate(C, a, b, hid, top);
                        }
                    }
        }
    return -1;
}

static int build(Circ *C, uint64_t T, uint64_t M, unsigned avail, int depth);

static int pair_tries = 0; /* step 5 below: how many of the best gate pairs to try (0 = off) */

/* Step 5: T = LUT(g1, g2, B) for two existing gates g1, g2 and one new
 * sub-circuit B.  Inside each of the four classes of (g1, g2) the LUT is a
 * function of B alone: a constant where T is constant on the class (B is
 * free there), else B or ~B (B must equal T or ~T there).  So B's care set is
 * the union of the classes where T is mixed; pairs that leave the fewest care
 * bits are tried, with every polarity choice per mixed class. */
static int pair_decomp(Circ *C, uint64_t T, uint64_t M, unsigned avail, int depth) {
    int n = C->n;
    enum { K = 6 };
    int best_a[K], best_b[K], cnt = 0;
    int best_c[K];
    for (int a = 0; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
            uint64_t care = 0;
            for (int q = 0; q < 4; ++q) {
                uint64_t cls = M & sel(C->g[a].tt, q & 2) & sel(C->g[b].tt, q & 1);
                uint64_t on = cls & T;
                if (on && on != cls) care |= cls;
            }
            int c = __builtin_popcountll(care);
            if (c == 0 || care == M) continue; /* no progress, or a plain LUT */
            /* keep the K smallest (random tie-break by replacing with prob 1/2) */
            int worst = -1;
            if (cnt < K) {
                worst = cnt++;
            } else {
                for (int i = 0; i < K; ++i)
                    if (worst < 0 || best_c[i] > best_c[worst]) worst = i;
                if (best_c[worst] < c || (best_c[worst] == c && (rnd() & 1))) worst = -1;
            }
            if (worst >= 0) {
                best_a[worst] = a;
                best_b[worst] = b;
                best_c[worst] = c;
            }
        }
    Circ best;
    int best_id = -1;
    int tries = cnt < pair_tries ? cnt : pair_tries;
    for (int t = 0; t < tries; ++t) {
        /* the t-th smallest */
        int pick = -1;
        for (int i = 0; i < cnt; ++i)
            if (best_c[i] >= 0 && (pick < 0 || best_c[i] < best_c[pick])) pick = i;
        if (pick < 0) break;
        int a = best_a[pick], b = best_b[pick];
        best_c[pick] = -1 - best_c[pick]; /* mark used */
        uint64_t quad[4];
        int mixed[4], nm = 0;
        for (int q = 0; q < 4; ++q) {
            quad[q] = M & sel(C->g[a].tt, q & 2) & sel(C->g[b].tt, q & 1);
            uint64_t on = quad[q] & T;
            if (on && on != quad[q]) mixed[nm++] = q;
        }
        for (int pol = 0; pol < (1 << (nm - 1)); ++pol) {
            uint64_t bt = 0, bm = 0;
            for (int m = 0; m < nm; ++m) {
                int q = mixed[m];
                int pq = m == 0 ? 0 : (pol >> (m - 1)) & 1;
                bt |= (pq ? ~T : T) & quad[q];
                bm |= quad[q];
            }
            Circ W = *C;
            int B = build(&W, bt, bm, avail, depth + 1);
            if (B < 0) continue;
            uint8_t lut;
            if (!fit3(W.g[a].tt, W.g[b].tt, W.g[B].tt, T, M, &lut)) continue;
            int id = add_gate(&W, a, b, B, lut);
            if (id < 0) continue;
            if (best_id < 0 || W.n < best.n) {
                best = W;
                best_id = id;
            }
        }
    }
    for (int i = 0; i < cnt; ++i)
        if (best_c[i] < 0) best_c[i] = -1 - best_c[i];
    if (best_id < 0) return -1;
    *C = best;
    return best_id;
}

/* Split on a random available variable; try the join variants and keep the
 * cheapest.  Returns the gate realising T on M, or -1. */
static int split(Circ *C, uint64_t T, uint64_t M, unsigned avail, int depth) {
    int vars[NIN], nv = 0;
    for (int v = 0; v < NIN; ++v)
        if ((avail >> v) & 1) vars[nv++] = v;
    if (nv == 0) return -1;
    Circ best;
    int best_id = -1;
    /* shallow nodes try every variable and join, deeper ones a random one */
    int wide = depth < wide_depth;
    int tries = wide ? nv : 1;
    for (int t = 0; t < tries; ++t) {
        int v = wide ? vars[t] : vars[rndn(nv)];
        uint64_t tv = C->g[v].tt;
        unsigned rest = avail & ~(1u << v);
        int allv = depth < variant_depth;
        int v0 = allv ? 0 : rndn(3), v1 = allv ? 3 : v0 + 1;
        for (int variant = v0; variant < v1; ++variant) {
            Circ W = *C;
            int id = -1;
            if (variant < 2) {
                /* variant 0: B targets T; variant 1: B targets T ^ A */
                int A = build(&W, T, M & ~tv, rest, depth + 1);
                if (A < 0) continue;
                uint64_t bt = variant == 0 ? T : (T ^ W.g[A].tt);
                int B = build(&W, bt, M & tv, rest, depth + 1);
                if (B < 0) continue;
                uint8_t lut;
                if (((W.g[A].tt ^ T) & M) == 0 || ((W.g[A].tt ^ T) & M) == M)
                    id = A;
                else if (fit3(tv, W.g[A].tt, W.g[B].tt, T, M, &lut))
                    id = add_gate(&W, v, A, B, lut);
            } else {
                /* variant 2: a second variable w with T|(v,w) a function of one signal X */
                int w = -1;
                int others[NIN], no = 0;
                for (int u = 0; u < NIN; ++u)
                    if (((rest >> u) & 1)) others[no++] = u;
                if (no == 0) continue;
                w = others[rndn(no)];
                uint64_t tw = C->g[w].tt;
                /* choose polarity per quadrant so X is consistent: X = T ^ pol_q on quadrant q */
                uint64_t quad[4];
                int nonconst[4], nnc = 0;
                for (int q = 0; q < 4; ++q) {
                    quad[q] = M & sel(tv, q & 2) & sel(tw, q & 1);
                    uint64_t on = quad[q] & T;
                    if (on != 0 && on != quad[q]) nonconst[nnc++] = q;
                }
                if (nnc == 0) continue;
                int best_local = -1;
                Circ bestW;
                for (int pol = 0; pol < (1 << (nnc - 1)); ++pol) { /* first quadrant fixed */
                    uint64_t xt = 0, xm = 0;
                    for (int m = 0; m < nnc; ++m) {
                        int q = nonconst[m];
                        int pq = m == 0 ? 0 : (pol >> (m - 1)) & 1;
                        xt |= (pq ? ~T : T) & quad[q];
                        xm |= quad[q];
                    }
                    Circ V = W;
                    int X = build(&V, xt, xm, rest & ~(1u << w), depth + 1);
                    if (X < 0) continue;
                    uint8_t lut;
                    int id2 = -1;
                    if (fit3(tv, tw, V.g[X].tt, T, M, &lut)) id2 = add_gate(&V, v, w, X, lut);
                    if (id2 < 0) continue;
                    if (best_local < 0 || V.n < bestW.n) {
                        bestW = V;
                        best_local = id2;
                    }
                }
                if (best_local < 0) continue;
                W = bestW;
                id = best_local;
            }
            if (id < 0) continue;
            if (best_id < 0 || W.n < best.n) {
                best = W;
                best_id = id;
            }
        }
    }
    if (pair_tries > 0 && depth < wide_depth + 2) {
        Circ W = *C;
        int id = pair_decomp(&W, T, M, avail, depth);
        if (id >= 0 && (best_id < 0 || W.n < best.n)) {
            best = W;
            best_id = id;
        }
    }
    if (best_id < 0) return -1;
    *C = best;
    return best_id;
}

static int build(Circ *C, uint64_t T, uint64_t M, unsigned avail, int depth) {
    int id = find_existing(C, T, M);
    if (id >= 0) return id;
    id = try_lut1(C, T, M);
    if (id >= 0) return id;
    if (C->n >= MAXG - 4) return -1;
    Circ W = *C;
    id = try_lut2(&W, T, M);
    if (id >= 0) {
        *C = W;
        return id;
    }
    return split(C, T, M, avail, depth);
}

static void init(Circ *C) {
    memset(C, 0, sizeof *C);
    for (int v = 0; v < NIN; ++v) {
        uint64_t t = 0;
        for (int x = 0; x < 64; ++x)
            if ((x >> (NIN - 1 - v)) & 1) t |= 1ULL << x;
        C->g[v].tt = t;
        C->g[v].in[0] = C->g[v].in[1] = C->g[v].in[2] = -1;
    }
    C->n = NIN;
}

int main(int argc, char **argv) {
    if (argc < 7) {
        fprintf(stderr, "usage: %s T0 T1 T2 T3 iterations seed [lut2_limit]\n", argv[0]);
        return 2;
    }
    uint64_t T[4];
    for (int t = 0; t < 4; ++t) T[t] = strtoull(argv[1 + t], NULL, 16);
    long iters = atol(argv[5]);
    rng_state = strtoull(argv[6], NULL, 10) * 0x9E3779B97F4A7C15ULL + 1;
    lut2_limit = argc > 7 ? atoi(argv[7]) : 0;
    wide_depth = argc > 8 ? atoi(argv[8]) : 1;
    variant_depth = argc > 9 ? atoi(argv[9]) : 99;
    pair_tries = argc > 10 ? atoi(argv[10]) : 0;

    Circ best;
    int have = 0;
    for (long it = 0; it < iters; ++it) {
        Circ C;
        init(&C);
        int order[4] = {0, 1, 2, 3};
        for (int i = 3; i > 0; --i) {
            int j = rndn(i + 1);
            int tmp = order[i];
            order[i] = order[j];
            order[j] = tmp;
        }
        int ok = 1;
        for (int k = 0; k < 4 && ok; ++k) {
            int t = order[k];
            int id = build(&C, T[t], ~0ULL, (1u << NIN) - 1, 0);
            if (id < 0) {
                ok = 0;
                break;
            }
            C.out[t] = id;
            C.neg[t] = (uint8_t)(C.g[id].tt != T[t]);
        }
        if (!ok) continue;
        if (!have || C.n < best.n) {
            best = C;
            have = 1;
            fprintf(stderr, "iter %ld: %d gates\n", it, C.n - NIN);
        }
    }
    if (!have) return 1;
    printf("gates %d\n", best.n - NIN);
    for (int i = NIN; i < best.n; ++i)
        printf("g %d %d %d %d %d\n", i, best.g[i].in[0], best.g[i].in[1], best.g[i].in[2],
               best.g[i].lut);
    for (int t = 0; t < 4; ++t) printf("out %d %d %d\n", t, best.out[t], best.neg[t]);
    return 0;
}
