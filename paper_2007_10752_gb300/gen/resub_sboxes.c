/*
 * resub_sboxes.c -- shrink a LOP3 circuit by resubstitution with
 * observability don't-cares (a post-pass for the circuits of sbox_search.c).
 *
 * For a gate g, its care set is the set of the 64 input points at which
 * complementing g changes some circuit output.  Outside it, g may take any
 * value.  g is replaced, on its care set, by
 *   (0) an existing signal or its complement,
 *   (1) one new LUT over three existing signals, or
 *   (2) LUT(a, b, h) with h a new LUT over three existing signals,
 * using only signals outside g's transitive fanout and outside its maximum
 * fanout-free cone (the gates that die with g).  That cone then dies, so the
 * circuit shrinks by its size minus the gates the replacement costs.  Passes
 * repeat until no replacement gains a gate.  The result is checked against
 * the outputs of the input circuit over all 64 points.
 *
 * Circuit text format (as sbox_search.c writes it): "g <id> <a> <b> <c> <lut>"
 * lines (signals 0..5 are the inputs, gate i is signal 6 + i, lut bit
 * (a << 2 | b << 1 | c)), then "out <t> <id> <neg>" for the 4 outputs.
 *
 * Usage: resub_sboxes < circuit.txt > smaller.txt
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXS 160
typedef uint64_t tt;

typedef struct {
    int ng;
    int a[MAXS], b[MAXS], c[MAXS];
    int lut[MAXS];
    int out[4], neg[4];
} circ_t;

static tt lut_eval(int lut, tt a, tt b, tt c) {
    tt r = 0;
    for (int i = 0; i < 8; ++i)
        if ((lut >> i) & 1) r |= ((i & 4) ? a : ~a) & ((i & 2) ? b : ~b) & ((i & 1) ? c : ~c);
    return r;
}

static void eval(const circ_t *k, tt *s) {
    for (int v = 0; v < 6; ++v) {
        tt t = 0;
        for (int x = 0; x < 64; ++x)
            if ((x >> (5 - v)) & 1) t |= (tt)1 << x;
        s[v] = t;
    }
    for (int i = 0; i < k->ng; ++i) s[6 + i] = lut_eval(k->lut[i], s[k->a[i]], s[k->b[i]], s[k->c[i]]);
}

static void outputs(const circ_t *k, const tt *s, tt *o) {
    for (int t = 0; t < 4; ++t) o[t] = s[k->out[t]] ^ (k->neg[t] ? ~(tt)0 : 0);
}

/* LUT over (x, y, z) equal to target on care, or -1 */
static int fit3(tt x, tt y, tt z, tt target, tt care) {
    int lut = 0;
    for (int i = 0; i < 8; ++i) {
        tt cls = ((i & 4) ? x : ~x) & ((i & 2) ? y : ~y) & ((i & 1) ? z : ~z) & care;
        tt on = cls & target;
        if (on) {
            if (on != cls) return -1;
            lut |= 1 << i;
        }
    }
    return lut;
}

/* care set of signal g: points where complementing it changes an output */
static tt care_of(const circ_t *k, const tt *s, int g) {
    tt t[MAXS + 6];
    memcpy(t, s, sizeof(tt) * (6 + k->ng));
    t[g] = ~t[g];
    for (int i = g - 6 + 1; i < k->ng; ++i)
        t[6 + i] = lut_eval(k->lut[i], t[k->a[i]], t[k->b[i]], t[k->c[i]]);
    tt o0[4], o1[4], care = 0;
    outputs(k, s, o0);
    outputs(k, t, o1);
    for (int q = 0; q < 4; ++q) care |= o0[q] ^ o1[q];
    return care;
}

/* tfo[v] = 1 for every signal in the transitive fanout of g (g included) */
static void tfo_of(const circ_t *k, int g, char *tfo) {
    memset(tfo, 0, MAXS + 6);
    tfo[g] = 1;
    for (int i = 0; i < k->ng; ++i)
        if (tfo[k->a[i]] || tfo[k->b[i]] || tfo[k->c[i]]) tfo[6 + i] = 1;
}

/* reference counts: fanouts plus circuit outputs */
static void refs_of(const circ_t *k, int *ref) {
    memset(ref, 0, sizeof(int) * (MAXS + 6));
    for (int i = 0; i < k->ng; ++i) {
        ref[k->a[i]]++;
        ref[k->b[i]]++;
        ref[k->c[i]]++;
    }
    for (int t = 0; t < 4; ++t) ref[k->out[t]]++;
}

/* maximum fanout-free cone of gate g: mark the gates that die with it */
static int mffc_mark(const circ_t *k, int *ref, int g, char *dead) {
    if (g < 6) return 0;
    dead[g] = 1;
    int n = 1, i = g - 6;
    int fi[3] = {k->a[i], k->b[i], k->c[i]};
    for (int q = 0; q < 3; ++q) {
        int v = fi[q];
        if (q == 1 && v == fi[0]) continue;
        if (q == 2 && (v == fi[0] || v == fi[1])) continue;
        if (v >= 6 && --ref[v] == 0) n += mffc_mark(k, ref, v, dead);
    }
    return n;
}

/* remove dead gates and restore a topological order after a rewrite */
static void compact(circ_t *k) {
    int n = 6 + k->ng;
    char live[MAXS + 6] = {0};
    /* liveness by reverse reachability from the outputs */
    int stack[MAXS + 6], sp = 0;
    for (int t = 0; t < 4; ++t)
        if (!live[k->out[t]]) { live[k->out[t]] = 1; stack[sp++] = k->out[t]; }
    while (sp) {
        int v = stack[--sp];
        if (v < 6) continue;
        int i = v - 6, fi[3] = {k->a[i], k->b[i], k->c[i]};
        for (int q = 0; q < 3; ++q)
            if (!live[fi[q]]) { live[fi[q]] = 1; stack[sp++] = fi[q]; }
    }
    /* topological order of live gates (Kahn) */
    int order[MAXS + 6], no = 0, placed[MAXS + 6] = {0};
    for (int v = 0; v < 6; ++v) placed[v] = 1;
    int progress = 1;
    while (progress) {
        progress = 0;
        for (int v = 6; v < n; ++v) {
            if (!live[v] || placed[v]) continue;
            int i = v - 6;
            if (placed[k->a[i]] && placed[k->b[i]] && placed[k->c[i]]) {
                placed[v] = 1;
                order[no++] = v;
                progress = 1;
            }
        }
    }
    int newid[MAXS + 6];
    for (int v = 0; v < 6; ++v) newid[v] = v;
    circ_t r;
    memset(&r, 0, sizeof r);
    for (int j = 0; j < no; ++j) newid[order[j]] = 6 + j;
    for (int j = 0; j < no; ++j) {
        int i = order[j] - 6;
        r.a[j] = newid[k->a[i]];
        r.b[j] = newid[k->b[i]];
        r.c[j] = newid[k->c[i]];
        r.lut[j] = k->lut[i];
    }
    r.ng = no;
    for (int t = 0; t < 4; ++t) {
        r.out[t] = newid[k->out[t]];
        r.neg[t] = k->neg[t];
    }
    *k = r;
}

/* replace every use of signal g by signal s (complemented if inv) */
static void rewire(circ_t *k, int g, int s, int inv) {
    for (int i = 0; i < k->ng; ++i) {
        int *fi[3] = {&k->a[i], &k->b[i], &k->c[i]};
        for (int q = 0; q < 3; ++q) {
            if (*fi[q] != g) continue;
            *fi[q] = s;
            if (inv) { /* complement input q of the LUT: swap the entries that differ in its bit */
                int bit = 4 >> q, l = k->lut[i], m = 0;
                for (int e = 0; e < 8; ++e)
                    if ((l >> (e ^ bit)) & 1) m |= 1 << e;
                k->lut[i] = m;
            }
        }
    }
    for (int t = 0; t < 4; ++t)
        if (k->out[t] == g) {
            k->out[t] = s;
            k->neg[t] ^= inv;
        }
}

/* one improving resubstitution, or 0 */
static int improve_once(circ_t *k) {
    tt s[MAXS + 6];
    eval(k, s);
    int n = 6 + k->ng;
    for (int g = n - 1; g >= 6; --g) {
        int ref[MAXS + 6];
        refs_of(k, ref);
        char dead[MAXS + 6] = {0}, tfo[MAXS + 6];
        int cone = mffc_mark(k, ref, g, dead);
        tfo_of(k, g, tfo);
        tt care = care_of(k, s, g);
        int cand[MAXS + 6], nc = 0;
        for (int v = 0; v < n; ++v)
            if (!tfo[v] && !dead[v]) cand[nc++] = v;
        /* (0) an existing signal */
        for (int j = 0; j < nc && cone >= 1; ++j) {
            tt d = (s[cand[j]] ^ s[g]) & care;
            if (d == 0 || d == care) {
                rewire(k, g, cand[j], d != 0);
                compact(k);
                return cone;
            }
        }
        /* (1) one LUT over three signals */
        if (cone >= 2)
            for (int x = 0; x < nc; ++x)
                for (int y = x + 1; y < nc; ++y)
                    for (int z = y + 1; z < nc; ++z) {
                        int l = fit3(s[cand[x]], s[cand[y]], s[cand[z]], s[g], care);
                        if (l < 0) continue;
                        int i = g - 6;
                        k->a[i] = cand[x];
                        k->b[i] = cand[y];
                        k->c[i] = cand[z];
                        k->lut[i] = l;
                        compact(k);
                        return cone - 1;
                    }
        /* (2) LUT(a, b, h), h = LUT(c, d, e) */
        if (cone >= 3)
            for (int x = 0; x < nc; ++x)
                for (int y = x + 1; y < nc; ++y) {
                    tt A = s[cand[x]], B = s[cand[y]];
                    tt cls[4] = {~A & ~B & care, ~A & B & care, A & ~B & care, A & B & care};
                    int var[4], nv = 0;
                    for (int q = 0; q < 4; ++q) {
                        tt on = cls[q] & s[g];
                        if (on && on != cls[q]) var[nv++] = q;
                    }
                    if (nv == 0) continue; /* a LUT of two signals: found by (1) */
                    tt hcare = 0;
                    for (int q = 0; q < nv; ++q) hcare |= cls[var[q]];
                    for (int pol = 0; pol < (1 << nv); ++pol) {
                        if (pol & 1) continue; /* h and ~h are the same gate */
                        tt target = 0;
                        for (int q = 0; q < nv; ++q)
                            target |= ((pol >> q) & 1 ? ~s[g] : s[g]) & cls[var[q]];
                        for (int c0 = 0; c0 < nc; ++c0)
                            for (int c1 = c0 + 1; c1 < nc; ++c1)
                                for (int c2 = c1 + 1; c2 < nc; ++c2) {
                                    int lh = fit3(s[cand[c0]], s[cand[c1]], s[cand[c2]], target, hcare);
                                    if (lh < 0) continue;
                                    tt H = lut_eval(lh, s[cand[c0]], s[cand[c1]], s[cand[c2]]);
                                    int lg = fit3(A, B, H, s[g], care);
                                    if (lg < 0) continue;
                                    int hi = k->ng++;
                                    k->a[hi] = cand[c0];
                                    k->b[hi] = cand[c1];
                                    k->c[hi] = cand[c2];
                                    k->lut[hi] = lh;
                                    int i = g - 6;
                                    k->a[i] = cand[x];
                                    k->b[i] = cand[y];
                                    k->c[i] = 6 + hi;
                                    k->lut[i] = lg;
                                    compact(k);
                                    return cone - 2;
                                }
                    }
                }
    }
    return 0;
}

int main(void) {
    circ_t k;
    memset(&k, 0, sizeof k);
    char line[256];
    while (fgets(line, sizeof line, stdin)) {
        int id, a, b, c, l, t, neg;
        if (sscanf(line, "g %d %d %d %d %d", &id, &a, &b, &c, &l) == 5) {
            if (id != 6 + k.ng || k.ng >= MAXS - 8) return 2;
            k.a[k.ng] = a;
            k.b[k.ng] = b;
            k.c[k.ng] = c;
            k.lut[k.ng] = l;
            k.ng++;
        } else if (sscanf(line, "out %d %d %d", &t, &id, &neg) == 3 && t >= 0 && t < 4) {
            k.out[t] = id;
            k.neg[t] = neg;
        }
    }
    tt s0[MAXS + 6], ref[4];
    eval(&k, s0);
    outputs(&k, s0, ref);
    int before = k.ng;
    while (improve_once(&k) > 0) {
    }
    tt s1[MAXS + 6], got[4];
    eval(&k, s1);
    outputs(&k, s1, got);
    for (int t = 0; t < 4; ++t)
        if (got[t] != ref[t]) {
            fprintf(stderr, "resub: output %d changed\n", t);
            return 1;
        }
    fprintf(stderr, "resub: %d -> %d gates\n", before, k.ng);
    for (int i = 0; i < k.ng; ++i) printf("g %d %d %d %d %d\n", 6 + i, k.a[i], k.b[i], k.c[i], k.lut[i]);
    for (int t = 0; t < 4; ++t) printf("out %d %d %d\n", t, k.out[t], k.neg[t]);
    return 0;
}
