/*
 * Seeded synthetic netlist generator.
 *
 * Produces the two text inputs that both the library and the CPU oracle read:
 *   - a cell library (13 combinational functions x drives X1/X2/X4, one DFF),
 *   - a levelized combinational netlist cut at flip-flops.
 *
 * The paper's designs (three proprietary netlists and seven IWLS 2005
 * benchmarks, Sec. V-A) are not available, so seeded random netlists with the
 * same structure stand in for them: startpoints are primary inputs plus DFF Q
 * pins (pseudo-primary inputs, Sec. III-A), DFF D pins are pseudo-primary
 * outputs, and every cell sits at an exact level.
 *
 * This module draws structure and capacitances only. It evaluates no logic,
 * probability, toggle rate or power: none of the method's arithmetic lives
 * here.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).
 *
 * Recipe (all draws from one SplitMix64 stream seeded with `seed`):
 *   1. Level 0 holds n_pi primary inputs, then n_dff DFF Q nets.
 *   2. Cells are split evenly over levels 1..depth (the first n_cells % depth
 *      levels get one extra cell).
 *   3. Each net draws a fanout budget from a geometric law on {1,2,...} with
 *      mean 2, capped at fanout_cap.
 *   4. Each cell draws its function uniformly from the 13 functions and its
 *      drive uniformly from X1/X2/X4. Its first fanin comes from level l-1
 *      (so its level is exact); each further fanin comes from level l-1 with
 *      probability p_prev, else from a uniform level in [0, l-2]. Within the
 *      source level a net is drawn uniformly, preferring nets with budget
 *      left, never a net already used by the same cell, and never a net at
 *      the fanout cap (the first fanin may exceed the cap only if all of
 *      level l-1 is at the cap). The fanins are then shuffled over the pins.
 *   5. Each DFF D pin is attached to a net drawn from the last 8 levels,
 *      preferring nets with no fanout yet.
 *   6. Nets that still have no fanout become primary outputs.
 *   7. Wire caps are uniform in [0.5, 2] fF, quantised to 1/4096 fF so that
 *      they are exact in binary32.
 *   8. With `shuffle`, net declarations and cell lines are written in a random
 *      order, so readers must not rely on file order being topological.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t seed;
    int64_t n_cells;
    int64_t n_pi;
    int64_t n_dff;
    int32_t depth;
    int32_t fanout_cap;
    double p_prev;
    int32_t shuffle;
} ng_params;

/* ---- SplitMix64 ---- */
static uint64_t sm64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double u01(uint64_t *s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }
static int64_t below(uint64_t *s, int64_t n) {
    if (n <= 0) return 0;
    return (int64_t)(((unsigned __int128)sm64(s) * (uint64_t)n) >> 64);
}

/* ---- the 13 library functions (name, output pin, input pins, expression) ---- */
typedef struct { const char *name; const char *out; int k; const char *pins[3]; const char *func; } fn_t;
static const fn_t FN[13] = {
    {"INV", "ZN", 1, {"A"}, "!A"},
    {"BUF", "Z", 1, {"A"}, "A"},
    {"NAND2", "ZN", 2, {"A1", "A2"}, "!(A1 & A2)"},
    {"NOR2", "ZN", 2, {"A1", "A2"}, "!(A1 | A2)"},
    {"AND2", "ZN", 2, {"A1", "A2"}, "A1 & A2"},
    {"OR2", "ZN", 2, {"A1", "A2"}, "A1 | A2"},
    {"XOR2", "Z", 2, {"A", "B"}, "A ^ B"},
    {"XNOR2", "ZN", 2, {"A", "B"}, "!(A ^ B)"},
    {"NAND3", "ZN", 3, {"A1", "A2", "A3"}, "!(A1 & A2 & A3)"},
    {"NOR3", "ZN", 3, {"A1", "A2", "A3"}, "!(A1 | A2 | A3)"},
    {"AOI21", "ZN", 3, {"A1", "A2", "B"}, "!((A1 & A2) | B)"},
    {"OAI21", "ZN", 3, {"A1", "A2", "B"}, "!((A1 | A2) & B)"},
    {"MUX2", "Z", 3, {"A", "B", "S"}, "(A & !S) | (B & S)"},
};
static const char *DRV[3] = {"X1", "X2", "X4"};
static const char *DRV_CAP[3] = {"0.8", "1.6", "3.2"};

/* ---- growable text buffer ---- */
typedef struct { char *p; size_t n, cap; int oom; } buf_t;
static void bput(buf_t *b, const char *s, size_t n) {
    if (b->oom) return;
    if (b->n + n + 1 > b->cap) {
        size_t c = b->cap ? b->cap : 1 << 16;
        while (c < b->n + n + 1) c *= 2;
        char *q = (char *)realloc(b->p, c);
        if (!q) { b->oom = 1; return; }
        b->p = q; b->cap = c;
    }
    memcpy(b->p + b->n, s, n);
    b->n += n;
    b->p[b->n] = 0;
}
static void bputs(buf_t *b, const char *s) { bput(b, s, strlen(s)); }
static void bputi(buf_t *b, int64_t v) { char t[32]; int n = snprintf(t, sizeof t, "%lld", (long long)v); bput(b, t, (size_t)n); }

char *ng_library_text(void) {
    buf_t b = {0};
    bputs(&b, "# synthetic 13-function library, drives X1/X2/X4\nlibrary synth13\n");
    for (int d = 0; d < 3; d++)
        for (int f = 0; f < 13; f++) {
            bputs(&b, "cell "); bputs(&b, FN[f].name); bputs(&b, "_"); bputs(&b, DRV[d]);
            bputs(&b, " "); bputs(&b, FN[f].out); bputs(&b, " "); bputs(&b, DRV_CAP[d]);
            bputs(&b, " "); bputs(&b, FN[f].func); bputs(&b, "\n");
        }
    bputs(&b, "seq DFF_X1 D Q 0.8\n");
    return b.oom ? (free(b.p), (char *)0) : b.p;
}

void ng_free(char *p) { free(p); }

/* Generates a netlist; returns 0 on success, else a negative code. */
int ng_generate(const ng_params *P, char **netlist_out, int64_t *n_nets_out) {
    *netlist_out = 0;
    if (P->depth < 1 || P->n_cells < 0 || P->n_pi < 0 || P->n_dff < 0 || P->fanout_cap < 1) return -1;
    if (P->n_pi + P->n_dff < 1 && P->n_cells > 0) return -1;
    if (P->n_cells > 0 && P->n_cells < P->depth) return -1;
    uint64_t rs = P->seed ^ 0x5DEECE66Dull;
    const int64_t ns = P->n_pi + P->n_dff, nc = P->n_cells, nn = ns + nc;
    const int L = P->depth, cap = P->fanout_cap;
    int64_t *lvl_start = (int64_t *)calloc((size_t)L + 2, sizeof(int64_t));
    int32_t *fanout = (int32_t *)calloc((size_t)(nn ? nn : 1), sizeof(int32_t));
    int32_t *budget = (int32_t *)calloc((size_t)(nn ? nn : 1), sizeof(int32_t));
    uint8_t *cfn = (uint8_t *)calloc((size_t)(nc ? nc : 1), 1);
    uint8_t *cdrv = (uint8_t *)calloc((size_t)(nc ? nc : 1), 1);
    int64_t *cin = (int64_t *)calloc((size_t)(nc ? nc : 1) * 3, sizeof(int64_t));
    int64_t *dffd = (int64_t *)calloc((size_t)(P->n_dff ? P->n_dff : 1), sizeof(int64_t));
    if (!lvl_start || !fanout || !budget || !cfn || !cdrv || !cin || !dffd) return -2;

    /* level l occupies nets [lvl_start[l], lvl_start[l+1]) */
    lvl_start[0] = 0;
    lvl_start[1] = ns;
    int64_t per = nc / L, extra = nc % L;
    for (int l = 1; l <= L; l++) lvl_start[l + 1] = lvl_start[l] + per + (l - 1 < extra ? 1 : 0);
    if (nc == 0) for (int l = 1; l <= L; l++) lvl_start[l + 1] = ns;
    for (int64_t n = 0; n < nn; n++) {
        int k = 1;
        while (k < cap && u01(&rs) < 0.5) k++;
        budget[n] = k;
    }

    for (int l = 1; l <= L && nc > 0; l++) {
        for (int64_t n = lvl_start[l]; n < lvl_start[l + 1]; n++) {
            int64_t c = n - ns;
            int f = (int)below(&rs, 13), k = FN[f].k;
            cfn[c] = (uint8_t)f;
            cdrv[c] = (uint8_t)below(&rs, 3);
            int64_t pick[3];
            for (int j = 0; j < k; j++) {
                int src = l - 1;
                if (j > 0 && l >= 2 && u01(&rs) >= P->p_prev) src = (int)below(&rs, l - 1);
                int64_t got = -1;
                /* try the drawn level, then fall back to l-1, then every lower level */
                for (int attempt = 0; attempt < l + 2 && got < 0; attempt++) {
                    int lv = attempt == 0 ? src : (attempt == 1 ? l - 1 : l - attempt);
                    if (lv < 0) break;
                    int64_t b0 = lvl_start[lv], cnt = lvl_start[lv + 1] - lvl_start[lv];
                    if (cnt <= 0) continue;
                    for (int pass = 0; pass < 3 && got < 0; pass++) {
                        int tries = pass < 2 ? 16 : 0;
                        for (int t = 0; t < tries && got < 0; t++) {
                            int64_t cand = b0 + below(&rs, cnt);
                            int dup = 0;
                            for (int i = 0; i < j; i++) dup |= pick[i] == cand;
                            if (dup || fanout[cand] >= cap) continue;
                            if (pass == 0 && fanout[cand] >= budget[cand]) continue;
                            got = cand;
                        }
                        if (pass == 2) {
                            int64_t st = below(&rs, cnt);
                            for (int64_t i = 0; i < cnt && got < 0; i++) {
                                int64_t cand = b0 + (st + i) % cnt;
                                int dup = 0;
                                for (int q = 0; q < j; q++) dup |= pick[q] == cand;
                                if (!dup && fanout[cand] < cap) got = cand;
                            }
                        }
                    }
                    if (j == 0) break; /* the first fanin must stay on level l-1 */
                }
                if (got < 0 && j == 0) { /* level l-1 saturated: exceed the cap to keep the level exact */
                    got = lvl_start[l - 1] + below(&rs, lvl_start[l] - lvl_start[l - 1]);
                }
                if (got < 0) { /* no distinct net left anywhere below: allow a repeated net */
                    got = pick[0];
                }
                pick[j] = got;
                fanout[got]++;
            }
            /* shuffle fanins over the pins */
            for (int j = k - 1; j > 0; j--) {
                int r = (int)below(&rs, j + 1);
                int64_t t = pick[j]; pick[j] = pick[r]; pick[r] = t;
            }
            for (int j = 0; j < 3; j++) cin[c * 3 + j] = j < k ? pick[j] : -1;
        }
    }
    /* DFF D pins: nets from the last 8 levels, preferring nets without fanout */
    int lo = L - 7 < 1 ? 1 : L - 7;
    int64_t dlo = nc > 0 ? lvl_start[lo] : 0, dcnt = nc > 0 ? lvl_start[L + 1] - lvl_start[lo] : ns;
    for (int64_t i = 0; i < P->n_dff; i++) {
        int64_t got = -1;
        for (int t = 0; t < 16 && got < 0; t++) {
            int64_t cand = dlo + below(&rs, dcnt);
            if (fanout[cand] == 0) got = cand;
        }
        for (int t = 0; t < 16 && got < 0; t++) {
            int64_t cand = dlo + below(&rs, dcnt);
            if (fanout[cand] < cap) got = cand;
        }
        if (got < 0) got = dlo + below(&rs, dcnt);
        dffd[i] = got;
        fanout[got]++;
    }

    /* output order of nets and cells */
    int64_t *net_order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn ? nn : 1));
    int64_t *cell_order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc ? nc : 1));
    if (!net_order || !cell_order) return -2;
    for (int64_t i = 0; i < nn; i++) net_order[i] = i;
    for (int64_t i = 0; i < nc; i++) cell_order[i] = i;
    if (P->shuffle) {
        for (int64_t i = nn - 1; i > 0; i--) { int64_t r = below(&rs, i + 1), t = net_order[i]; net_order[i] = net_order[r]; net_order[r] = t; }
        for (int64_t i = nc - 1; i > 0; i--) { int64_t r = below(&rs, i + 1), t = cell_order[i]; cell_order[i] = cell_order[r]; cell_order[r] = t; }
    }

    buf_t b = {0};
    bputs(&b, "# synthetic netlist: seed "); bputi(&b, (int64_t)P->seed);
    bputs(&b, ", cells "); bputi(&b, nc); bputs(&b, ", depth "); bputi(&b, L); bputs(&b, "\n");
    bputs(&b, "design synth_"); bputi(&b, (int64_t)P->seed); bputs(&b, "\n");
    for (int64_t i = 0; i < nn; i++) {
        int64_t n = net_order[i];
        /* wire cap U[0.5, 2] fF on a 1/4096 fF grid */
        int64_t q = 2048 + below(&rs, 6145);
        char t[64];
        int len = snprintf(t, sizeof t, "net n%lld %.12g\n", (long long)n, (double)q / 4096.0);
        bput(&b, t, (size_t)len);
    }
    for (int64_t i = 0; i < P->n_pi; i++) { bputs(&b, "input n"); bputi(&b, i); bputs(&b, "\n"); }
    for (int64_t i = 0; i < P->n_dff; i++) {
        bputs(&b, "dff r"); bputi(&b, i); bputs(&b, " DFF_X1 D=n"); bputi(&b, dffd[i]);
        bputs(&b, " Q=n"); bputi(&b, P->n_pi + i); bputs(&b, "\n");
    }
    for (int64_t i = 0; i < nc; i++) {
        int64_t c = cell_order[i];
        const fn_t *f = &FN[cfn[c]];
        bputs(&b, "cell u"); bputi(&b, c); bputs(&b, " "); bputs(&b, f->name); bputs(&b, "_"); bputs(&b, DRV[cdrv[c]]);
        for (int j = 0; j < f->k; j++) { bputs(&b, " "); bputs(&b, f->pins[j]); bputs(&b, "=n"); bputi(&b, cin[c * 3 + j]); }
        bputs(&b, " "); bputs(&b, f->out); bputs(&b, "=n"); bputi(&b, ns + c); bputs(&b, "\n");
    }
    for (int64_t n = ns; n < nn; n++)
        if (fanout[n] == 0) { bputs(&b, "output n"); bputi(&b, n); bputs(&b, "\n"); }

    free(lvl_start); free(fanout); free(budget); free(cfn); free(cdrv); free(cin); free(dffd);
    free(net_order); free(cell_order);
    if (b.oom) { free(b.p); return -2; }
    *netlist_out = b.p;
    if (n_nets_out) *n_nets_out = nn;
    return 0;
}
