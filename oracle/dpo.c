/*
 * DiffPower FP64 CPU oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct restatement of what DiffPower
 * (arXiv 2608.03778) computes, used to check the GPU library.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or helper with the GPU library and
 * neither includes nor calls it.  All floating point is binary64.
 *
 * Equation numbers follow the order of appearance in the paper:
 *   Eq. 1 switching power, Eq. 2 TR_model, Eq. 3 P_virus, Eq. 4 TR_acc,
 *   Eq. 5 beta, Eq. 6 beta-scaled gradient, Eq. 7 gradient accumulation,
 *   Eq. 8 sizing score, Eq. 9 power-virus proxy.
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *   - A cell's SP is the multilinear extension of its truth table
 *     (sum over input minterms of f(m) * prod_i (m_i ? a_i : 1 - a_i)); this is
 *     the exact SP under input independence and equals the paper's stack
 *     interpreter (Algorithm 2) on every read-once expression.
 *   - 1 - P of a net is evaluated as P(net = 0) under the same independence
 *     model (sum over the minterms where f is 0), never as 1 minus a rounded
 *     P: many nets of deep netlists sit within 1e-15 of 0 or 1, where the
 *     subtraction would lose all relative accuracy of TR_model = 2P(1-P)
 *     (Eq. 2) and could even make it negative.
 *   - Startpoint TR is the given input TR (tr_mode 0) or 2P(1-P) (tr_mode 1).
 *   - Local gradient term: d(K C (2P(1-P)))/dP = K C (2 - 4P) (Sec. III-E).
 *   - Hybrid gradient modes: 1 = paper (the accumulated gradient of each net is
 *     multiplied by its beta, Eq. 6); 2 = exact gradient of the hybrid power
 *     with beta held fixed.
 *   - Simulation: bit b of word t is lane b at cycle t; 64 independent Markov
 *     chains per startpoint; Philox4x32-10 counter (stream, t / 2, b mod 16, 0),
 *     output component b / 16, whose low 16 bits drive even cycles and high
 *     16 bits odd cycles; thresholds floor(p * 2^16) in binary64.
 *   - beta when TR_model = 0: 1 if TR_acc = 0, else beta_max.
 *
 * Pins (what fixes each function independently of itself) are in the tests:
 *   per-gate SP and partials: closed forms; forward on fanout-free circuits:
 *   brute-force enumeration; forward on any circuit with 0/1 inputs: Boolean
 *   evaluation; gradients: central finite differences and linearity in the
 *   caps; simulation: Boolean evaluation of the words, Markov statistics and
 *   generator statistics; beta-scaled gradient (mode 1): closed form on
 *   chains; Philox: its published round function is pinned only by statistics
 *   and by agreement with the GPU (no known-answer vectors in the repository).
 */
#include <ctype.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_IN 16

/* ------------------------------------------------------------------ */
/* string -> id hash map (open addressing, FNV-1a)                    */
/* ------------------------------------------------------------------ */
typedef struct {
    char **key;
    int64_t *val;
    int64_t cap;
    int64_t n;
} Map;

static uint64_t fnv(const char *s, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; i++) { h ^= (unsigned char)s[i]; h *= 1099511628211ull; }
    return h;
}
static int map_init(Map *m, int64_t cap) {
    m->cap = 16;
    while (m->cap < 2 * cap + 16) m->cap *= 2;
    m->key = (char **)calloc((size_t)m->cap, sizeof(char *));
    m->val = (int64_t *)calloc((size_t)m->cap, sizeof(int64_t));
    m->n = 0;
    return m->key && m->val ? 0 : -1;
}
static void map_free(Map *m) {
    if (m->key) for (int64_t i = 0; i < m->cap; i++) free(m->key[i]);
    free(m->key); free(m->val);
    m->key = 0; m->val = 0;
}
static int map_grow(Map *m) {
    Map g;
    if (map_init(&g, m->cap) != 0) return -1;
    for (int64_t i = 0; i < m->cap; i++)
        if (m->key[i]) {
            uint64_t h = fnv(m->key[i], strlen(m->key[i])) & (uint64_t)(g.cap - 1);
            while (g.key[h]) h = (h + 1) & (uint64_t)(g.cap - 1);
            g.key[h] = m->key[i]; g.val[h] = m->val[i]; g.n++;
        }
    free(m->key); free(m->val);
    *m = g;
    return 0;
}
static int64_t map_get(const Map *m, const char *s, size_t n) {
    uint64_t h = fnv(s, n) & (uint64_t)(m->cap - 1);
    while (m->key[h]) {
        if (strlen(m->key[h]) == n && memcmp(m->key[h], s, n) == 0) return m->val[h];
        h = (h + 1) & (uint64_t)(m->cap - 1);
    }
    return -1;
}
/* returns 1 if inserted, 0 if present, -1 on allocation failure */
static int map_put(Map *m, const char *s, size_t n, int64_t v) {
    if (map_get(m, s, n) >= 0) return 0;
    if (2 * (m->n + 1) > m->cap && map_grow(m) != 0) return -1;
    uint64_t h = fnv(s, n) & (uint64_t)(m->cap - 1);
    while (m->key[h]) h = (h + 1) & (uint64_t)(m->cap - 1);
    m->key[h] = (char *)malloc(n + 1);
    if (!m->key[h]) return -1;
    memcpy(m->key[h], s, n); m->key[h][n] = 0;
    m->val[h] = v; m->n++;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Boolean expression evaluation, straight from the string.           */
/* Precedence NOT > AND > XOR > OR (Sec. III-A).                      */
/* ------------------------------------------------------------------ */
typedef struct {
    const char *p;
    int npin;
    char pin[ORC_MAX_IN][32];
    int val[ORC_MAX_IN];
    int err;
} Ev;

static void ev_ws(Ev *e) { while (*e->p == ' ' || *e->p == '\t') e->p++; }
static int ev_or(Ev *e);
static int ev_primary(Ev *e) {
    ev_ws(e);
    char c = *e->p;
    if (c == '(') {
        e->p++;
        int v = ev_or(e);
        ev_ws(e);
        if (*e->p != ')') { e->err = 1; return 0; }
        e->p++;
        return v;
    }
    if (c == '0' || c == '1') { e->p++; return c == '1'; }
    if (isalpha((unsigned char)c) || c == '_') {
        const char *s = e->p;
        while (isalnum((unsigned char)*e->p) || *e->p == '_') e->p++;
        size_t n = (size_t)(e->p - s);
        for (int i = 0; i < e->npin; i++)
            if (strlen(e->pin[i]) == n && memcmp(e->pin[i], s, n) == 0) return e->val[i];
        e->err = 2;
        return 0;
    }
    e->err = 3;
    return 0;
}
static int ev_unary(Ev *e) {
    ev_ws(e);
    if (*e->p == '!' || *e->p == '~') { e->p++; return !ev_unary(e); }
    int v = ev_primary(e);
    ev_ws(e);
    while (*e->p == '\'') { e->p++; v = !v; ev_ws(e); }
    return v;
}
static int ev_and(Ev *e) {
    int v = ev_unary(e);
    for (;;) {
        ev_ws(e);
        if (*e->p == '&' || *e->p == '*') { e->p++; int w = ev_unary(e); v = v && w; }
        else return v;
    }
}
static int ev_xor(Ev *e) {
    int v = ev_and(e);
    for (;;) {
        ev_ws(e);
        if (*e->p == '^') { e->p++; int w = ev_and(e); v = v != w; }
        else return v;
    }
}
static int ev_or(Ev *e) {
    int v = ev_xor(e);
    for (;;) {
        ev_ws(e);
        if (*e->p == '|' || *e->p == '+') { e->p++; int w = ev_xor(e); v = v || w; }
        else return v;
    }
}

/* ------------------------------------------------------------------ */
/* library and netlist                                                 */
/* ------------------------------------------------------------------ */
typedef struct {
    char name[64];
    int seq;                      /* 1 = flip-flop (D pin is a pseudo-primary output) */
    char out[32];                 /* combinational output pin, or Q for a flop */
    char dpin[32];
    int k;                        /* number of inputs */
    char pin[ORC_MAX_IN][32];     /* input pins in order of first appearance */
    unsigned char *tt;            /* tt[m], bit i of m = value of pin[i] */
    double pincap;                /* fF, every input pin */
} LibCell;

typedef struct {
    int nlib;
    LibCell *lib;
    /* nets, in declaration order */
    int64_t nn;
    double *wire;
    int64_t *drv;       /* driving cell, or -1 for a startpoint, -2 if undriven */
    int64_t *start_of;  /* startpoint index, or -1 */
    double *ppo_cap;    /* total DFF D pin cap on the net */
    /* startpoints, in order of appearance (input lines and dff lines) */
    int64_t ns;
    int64_t *start_net;
    /* cells, in order of appearance */
    int64_t nc;
    int *cell_lib;
    int64_t *cell_out;
    int64_t *fin_ptr;   /* fanins of cell c: fin_net[fin_ptr[c] .. fin_ptr[c+1]) in lib pin order */
    int64_t *fin_net;
    double *pincap;
    /* sinks of each net (cell, pin) in cell order */
    int64_t *sink_ptr;
    int64_t *sink_cell;
    int64_t *topo;      /* cells in a topological order (Kahn) */
    int32_t depth;
    /* cells by level (1 + the deepest fanin's level), for the level-parallel CPU baseline:
     * level l holds lvl_cell[lvl_ptr[l - 1] .. lvl_ptr[l]), in cell order */
    int64_t *lvl_ptr;
    int64_t *lvl_cell;
} Orc;

static void orc_destroy(Orc *o) {
    if (!o) return;
    for (int i = 0; i < o->nlib; i++) free(o->lib[i].tt);
    free(o->lib); free(o->wire); free(o->drv); free(o->start_of); free(o->ppo_cap);
    free(o->start_net); free(o->cell_lib); free(o->cell_out); free(o->fin_ptr); free(o->fin_net);
    free(o->pincap); free(o->sink_ptr); free(o->sink_cell); free(o->topo);
    free(o->lvl_ptr); free(o->lvl_cell);
    free(o);
}

void orc_free(void *h) { orc_destroy((Orc *)h); }

static void seterr(char *err, int errlen, const char *msg, int64_t line) {
    if (err && errlen > 0) snprintf(err, (size_t)errlen, "%s (line %lld)", msg, (long long)line);
}

/* split the next line into whitespace tokens; returns the number of tokens */
static int tokens(const char **cur, char *linebuf, size_t cap, char **tok, int maxtok, const char **rest_after2) {
    const char *s = *cur;
    if (!*s) return -1;
    const char *e = strchr(s, '\n');
    size_t n = e ? (size_t)(e - s) : strlen(s);
    *cur = e ? e + 1 : s + n;
    if (n >= cap) n = cap - 1;
    memcpy(linebuf, s, n);
    linebuf[n] = 0;
    char *h = strchr(linebuf, '#');
    if (h) *h = 0;
    int nt = 0;
    char *p = linebuf;
    if (rest_after2) *rest_after2 = 0;
    while (*p && nt < maxtok) {
        while (*p == ' ' || *p == '\t' || *p == '\r') p++;
        if (!*p) break;
        tok[nt++] = p;
        while (*p && *p != ' ' && *p != '\t' && *p != '\r') p++;
        if (*p) *p++ = 0;
        if (nt == 4 && rest_after2) { while (*p == ' ' || *p == '\t') p++; *rest_after2 = p; }
    }
    return nt;
}

static int parse_library(Orc *o, const char *text, char *err, int errlen) {
    const char *cur = text;
    char line[4096];
    char *tok[8];
    int cap = 16;
    o->lib = (LibCell *)calloc((size_t)cap, sizeof(LibCell));
    if (!o->lib) return -1;
    int64_t ln = 0;
    for (;;) {
        const char *rest = 0;
        int nt = tokens(&cur, line, sizeof line, tok, 4, &rest);
        if (nt < 0) break;
        ln++;
        if (nt == 0 || strcmp(tok[0], "library") == 0) continue;
        if (o->nlib == cap) {
            cap *= 2;
            LibCell *q = (LibCell *)realloc(o->lib, sizeof(LibCell) * (size_t)cap);
            if (!q) return -1;
            o->lib = q;
        }
        LibCell *c = &o->lib[o->nlib];
        memset(c, 0, sizeof *c);
        if (strcmp(tok[0], "seq") == 0) {
            /* seq <ref> <d_pin> <q_pin> <d_pincap> */
            if (nt < 4 || !rest || !*rest) { seterr(err, errlen, "bad seq line", ln); return -2; }
            c->seq = 1;
            snprintf(c->name, sizeof c->name, "%s", tok[1]);
            snprintf(c->dpin, sizeof c->dpin, "%s", tok[2]);
            snprintf(c->out, sizeof c->out, "%s", tok[3]);
            c->pincap = strtod(rest, 0);
            o->nlib++;
            continue;
        }
        if (strcmp(tok[0], "cell") != 0 || nt < 4 || !rest) { seterr(err, errlen, "bad library line", ln); return -2; }
        /* cell <ref> <out_pin> <pincap> <function ...> */
        snprintf(c->name, sizeof c->name, "%s", tok[1]);
        snprintf(c->out, sizeof c->out, "%s", tok[2]);
        c->pincap = strtod(tok[3], 0);
        const char *f = rest;
        /* input pins: identifiers in order of first appearance */
        for (const char *p = f; *p;) {
            if (isalpha((unsigned char)*p) || *p == '_') {
                const char *s = p;
                while (isalnum((unsigned char)*p) || *p == '_') p++;
                size_t n = (size_t)(p - s);
                int seen = 0;
                for (int i = 0; i < c->k; i++) seen |= strlen(c->pin[i]) == n && memcmp(c->pin[i], s, n) == 0;
                if (!seen) {
                    if (c->k == ORC_MAX_IN || n >= 32) { seterr(err, errlen, "too many or too long pins", ln); return -2; }
                    memcpy(c->pin[c->k], s, n); c->pin[c->k][n] = 0; c->k++;
                }
            } else p++;
        }
        int64_t M = (int64_t)1 << c->k;
        c->tt = (unsigned char *)malloc((size_t)M);
        if (!c->tt) return -1;
        for (int64_t m = 0; m < M; m++) {
            Ev e;
            memset(&e, 0, sizeof e);
            e.p = f;
            e.npin = c->k;
            for (int i = 0; i < c->k; i++) { memcpy(e.pin[i], c->pin[i], 32); e.val[i] = (int)((m >> i) & 1); }
            int v = ev_or(&e);
            ev_ws(&e);
            if (e.err || *e.p) { seterr(err, errlen, "bad function", ln); return -2; }
            c->tt[m] = (unsigned char)v;
        }
        o->nlib++;
    }
    return 0;
}

static int find_lib(const Orc *o, const char *name) {
    for (int i = 0; i < o->nlib; i++) if (strcmp(o->lib[i].name, name) == 0) return i;
    return -1;
}

void *orc_load(const char *netlist, const char *library, char *err, int errlen) {
    Orc *o = (Orc *)calloc(1, sizeof(Orc));
    if (!o) return 0;
    int rc = parse_library(o, library, err, errlen);
    if (rc != 0) { if (rc == -1) seterr(err, errlen, "out of memory", 0); orc_destroy(o); return 0; }

    /* pass 1: count */
    int64_t nnet = 0, ncell = 0, nstart = 0, nedge = 0, nlines = 0;
    for (const char *p = netlist; *p;) {
        const char *e = strchr(p, '\n');
        size_t n = e ? (size_t)(e - p) : strlen(p);
        while (n && (*p == ' ' || *p == '\t')) { p++; n--; }
        if (n >= 4 && memcmp(p, "net ", 4) == 0) nnet++;
        else if (n >= 5 && memcmp(p, "cell ", 5) == 0) {
            ncell++;
            for (size_t i = 0; i < n; i++) nedge += p[i] == '=';
        } else if (n >= 6 && memcmp(p, "input ", 6) == 0) nstart++;
        else if (n >= 4 && memcmp(p, "dff ", 4) == 0) nstart++;
        nlines++;
        p = e ? e + 1 : p + n;
    }
    o->nn = nnet; o->nc = ncell;
    size_t a = (size_t)(nnet + 1), b = (size_t)(ncell + 1);
    o->wire = (double *)calloc(a, sizeof(double));
    o->drv = (int64_t *)malloc(a * sizeof(int64_t));
    o->start_of = (int64_t *)malloc(a * sizeof(int64_t));
    o->ppo_cap = (double *)calloc(a, sizeof(double));
    o->start_net = (int64_t *)malloc((size_t)(nstart + 1) * sizeof(int64_t));
    o->cell_lib = (int *)malloc(b * sizeof(int));
    o->cell_out = (int64_t *)malloc(b * sizeof(int64_t));
    o->fin_ptr = (int64_t *)calloc(b, sizeof(int64_t));
    o->fin_net = (int64_t *)malloc((size_t)(nedge + 1) * sizeof(int64_t));
    o->pincap = (double *)malloc(b * sizeof(double));
    Map nets;
    if (!o->wire || !o->drv || !o->start_of || !o->ppo_cap || !o->start_net || !o->cell_lib || !o->cell_out ||
        !o->fin_ptr || !o->fin_net || !o->pincap || map_init(&nets, nnet) != 0) {
        seterr(err, errlen, "out of memory", 0); orc_destroy(o); return 0;
    }
    for (int64_t i = 0; i <= nnet; i++) { o->drv[i] = -2; o->start_of[i] = -1; }

    /* pass 2: parse */
    const char *cur = netlist;
    char *line = (char *)malloc(1 << 16);
    char *tok[4 + 2 * ORC_MAX_IN];
    int64_t ln = 0, nets_seen = 0, cells_seen = 0, edges = 0;
    int fail = 0;
    while (!fail) {
        int nt = tokens(&cur, line, 1 << 16, tok, 4 + 2 * ORC_MAX_IN, 0);
        if (nt < 0) break;
        ln++;
        if (nt == 0 || strcmp(tok[0], "design") == 0) continue;
        if (strcmp(tok[0], "net") == 0) {
            if (nt != 3) { seterr(err, errlen, "bad net line", ln); fail = 1; break; }
            int r = map_put(&nets, tok[1], strlen(tok[1]), nets_seen);
            if (r == 0) { seterr(err, errlen, "net declared twice", ln); fail = 1; break; }
            if (r < 0) { seterr(err, errlen, "out of memory", ln); fail = 1; break; }
            o->wire[nets_seen] = strtod(tok[2], 0);
            nets_seen++;
        } else if (strcmp(tok[0], "input") == 0) {
            int64_t n = nt == 2 ? map_get(&nets, tok[1], strlen(tok[1])) : -1;
            if (n < 0 || o->drv[n] != -2) { seterr(err, errlen, "bad input line", ln); fail = 1; break; }
            o->drv[n] = -1; o->start_of[n] = o->ns; o->start_net[o->ns++] = n;
        } else if (strcmp(tok[0], "output") == 0) {
            if (nt != 2 || map_get(&nets, tok[1], strlen(tok[1])) < 0) { seterr(err, errlen, "bad output line", ln); fail = 1; break; }
        } else if (strcmp(tok[0], "dff") == 0) {
            int li = nt == 5 ? find_lib(o, tok[2]) : -1;
            if (li < 0 || !o->lib[li].seq) { seterr(err, errlen, "bad dff line", ln); fail = 1; break; }
            int64_t dn = -1, qn = -1;
            for (int t = 3; t < 5; t++) {
                char *eq = strchr(tok[t], '=');
                if (!eq) break;
                *eq = 0;
                int64_t n = map_get(&nets, eq + 1, strlen(eq + 1));
                if (strcmp(tok[t], o->lib[li].dpin) == 0) dn = n;
                else if (strcmp(tok[t], o->lib[li].out) == 0) qn = n;
            }
            if (dn < 0 || qn < 0 || o->drv[qn] != -2) { seterr(err, errlen, "bad dff pins", ln); fail = 1; break; }
            o->ppo_cap[dn] += o->lib[li].pincap;
            o->drv[qn] = -1; o->start_of[qn] = o->ns; o->start_net[o->ns++] = qn;
        } else if (strcmp(tok[0], "cell") == 0) {
            int li = nt >= 3 ? find_lib(o, tok[2]) : -1;
            if (li < 0 || o->lib[li].seq) { seterr(err, errlen, "unknown cell type", ln); fail = 1; break; }
            const LibCell *L = &o->lib[li];
            if (nt != 3 + L->k + 1) { seterr(err, errlen, "wrong pin count", ln); fail = 1; break; }
            int64_t c = cells_seen++;
            o->cell_lib[c] = li;
            o->pincap[c] = L->pincap;
            o->fin_ptr[c] = edges;
            int64_t outn = -1;
            int got[ORC_MAX_IN] = {0};
            for (int t = 3; t < nt; t++) {
                char *eq = strchr(tok[t], '=');
                if (!eq) { fail = 1; break; }
                *eq = 0;
                int64_t n = map_get(&nets, eq + 1, strlen(eq + 1));
                if (n < 0) { fail = 1; break; }
                if (strcmp(tok[t], L->out) == 0) { if (outn >= 0) { fail = 1; break; } outn = n; continue; }
                int pi = -1;
                for (int i = 0; i < L->k; i++) if (strcmp(L->pin[i], tok[t]) == 0) pi = i;
                if (pi < 0 || got[pi]) { fail = 1; break; }
                got[pi] = 1;
                o->fin_net[edges + pi] = n;
            }
            if (fail || outn < 0 || o->drv[outn] != -2) { seterr(err, errlen, "bad cell pins or multiple drivers", ln); fail = 1; break; }
            o->drv[outn] = c;
            o->cell_out[c] = outn;
            edges += L->k;
        } else {
            seterr(err, errlen, "unknown statement", ln); fail = 1;
        }
    }
    free(line);
    map_free(&nets);
    if (fail) { orc_destroy(o); return 0; }
    o->nc = cells_seen;
    o->fin_ptr[o->nc] = edges;
    for (int64_t n = 0; n < o->nn; n++)
        if (o->drv[n] == -2) { seterr(err, errlen, "undriven net", 0); orc_destroy(o); return 0; }

    /* sinks of every net, in cell order */
    o->sink_ptr = (int64_t *)calloc((size_t)o->nn + 1, sizeof(int64_t));
    o->sink_cell = (int64_t *)malloc((size_t)(edges + 1) * sizeof(int64_t));
    o->topo = (int64_t *)malloc((size_t)(o->nc + 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)o->nn + 1, sizeof(int64_t));
    int64_t *indeg = (int64_t *)calloc((size_t)o->nc + 1, sizeof(int64_t));
    int32_t *lev = (int32_t *)calloc((size_t)o->nn + 1, sizeof(int32_t));
    if (!o->sink_ptr || !o->sink_cell || !o->topo || !fill || !indeg || !lev) {
        free(fill); free(indeg); free(lev); seterr(err, errlen, "out of memory", 0); orc_destroy(o); return 0;
    }
    for (int64_t e = 0; e < edges; e++) o->sink_ptr[o->fin_net[e] + 1]++;
    for (int64_t n = 0; n < o->nn; n++) o->sink_ptr[n + 1] += o->sink_ptr[n];
    for (int64_t c = 0; c < o->nc; c++)
        for (int64_t e = o->fin_ptr[c]; e < o->fin_ptr[c + 1]; e++) {
            int64_t n = o->fin_net[e];
            o->sink_cell[o->sink_ptr[n] + fill[n]++] = c;
            if (o->drv[n] >= 0) indeg[c]++;
        }
    /* Kahn's algorithm */
    int64_t head = 0, tail = 0;
    for (int64_t c = 0; c < o->nc; c++) if (indeg[c] == 0) o->topo[tail++] = c;
    o->depth = 0;
    while (head < tail) {
        int64_t c = o->topo[head++];
        int32_t l = 0;
        for (int64_t e = o->fin_ptr[c]; e < o->fin_ptr[c + 1]; e++) if (lev[o->fin_net[e]] > l) l = lev[o->fin_net[e]];
        lev[o->cell_out[c]] = l + 1;
        if (l + 1 > o->depth) o->depth = l + 1;
        int64_t n = o->cell_out[c];
        for (int64_t s = o->sink_ptr[n]; s < o->sink_ptr[n + 1]; s++)
            if (--indeg[o->sink_cell[s]] == 0) o->topo[tail++] = o->sink_cell[s];
    }
    if (tail != o->nc) { free(fill); free(indeg); free(lev); seterr(err, errlen, "combinational cycle", 0); orc_destroy(o); return 0; }
    /* level buckets (counting sort by level, stable in cell order) */
    o->lvl_ptr = (int64_t *)calloc((size_t)o->depth + 2, sizeof(int64_t));
    o->lvl_cell = (int64_t *)malloc((size_t)(o->nc + 1) * sizeof(int64_t));
    if (!o->lvl_ptr || !o->lvl_cell) {
        free(fill); free(indeg); free(lev); seterr(err, errlen, "out of memory", 0); orc_destroy(o); return 0;
    }
    for (int64_t c = 0; c < o->nc; c++) o->lvl_ptr[lev[o->cell_out[c]]]++;
    for (int32_t l = 1; l <= o->depth; l++) o->lvl_ptr[l] += o->lvl_ptr[l - 1];
    for (int64_t c = o->nc - 1; c >= 0; c--) o->lvl_cell[--o->lvl_ptr[lev[o->cell_out[c]]]] = c;
    /* now lvl_ptr[l] = first cell of level l; shift so level l spans [lvl_ptr[l-1], lvl_ptr[l]) */
    for (int32_t l = 0; l < o->depth; l++) o->lvl_ptr[l] = o->lvl_ptr[l + 1];
    o->lvl_ptr[o->depth] = o->nc;
    free(fill); free(indeg); free(lev);
    return o;
}

void orc_info(const void *h, int64_t *out5) {
    const Orc *o = (const Orc *)h;
    out5[0] = o->nn; out5[1] = o->ns; out5[2] = o->nc; out5[3] = o->fin_ptr[o->nc]; out5[4] = o->depth;
}

/* net declaration index of each startpoint / each cell output */
void orc_start_nets(const void *h, int64_t *out) { const Orc *o = (const Orc *)h; memcpy(out, o->start_net, sizeof(int64_t) * (size_t)o->ns); }
void orc_cell_outs(const void *h, int64_t *out) { const Orc *o = (const Orc *)h; memcpy(out, o->cell_out, sizeof(int64_t) * (size_t)o->nc); }

void orc_set_pincap(void *h, int64_t cell, double cap) {
    Orc *o = (Orc *)h;
    if (cell >= 0 && cell < o->nc) o->pincap[cell] = cap;
}

/* Eq. 1: C_load of a net = wire cap + input pin caps of the cells it drives
 * (+ DFF D pin caps, the pseudo-primary outputs of Sec. III-A). */
void orc_cload(const void *h, double *cl) {
    const Orc *o = (const Orc *)h;
    for (int64_t n = 0; n < o->nn; n++) {
        double c = o->wire[n] + o->ppo_cap[n];
        for (int64_t s = o->sink_ptr[n]; s < o->sink_ptr[n + 1]; s++) c += o->pincap[o->sink_cell[s]];
        cl[n] = c;
    }
}

/* Probability that a cell's output is v (v = 1: its SP) under input independence:
 * sum over the input minterms m with f(m) = v of prod_i P(input i = m_i), where
 * P(input i = 1) = a1[i] and P(input i = 0) = a0[i]. */
static double cell_prob(const LibCell *L, const double *a1, const double *a0, int v) {
    int64_t M = (int64_t)1 << L->k;
    double s = 0.0;
    for (int64_t m = 0; m < M; m++) {
        if (L->tt[m] != v) continue;
        double p = 1.0;
        for (int i = 0; i < L->k; i++) p *= ((m >> i) & 1) ? a1[i] : a0[i];
        s += p;
    }
    return s;
}

/* d SP / d a_j of the same extension: sum_m f(m) (m_j ? 1 : -1) prod_{i != j}(...). */
static double cell_dsp(const LibCell *L, const double *a1, const double *a0, int j) {
    int64_t M = (int64_t)1 << L->k;
    double s = 0.0;
    for (int64_t m = 0; m < M; m++) {
        if (!L->tt[m]) continue;
        double p = ((m >> j) & 1) ? 1.0 : -1.0;
        for (int i = 0; i < L->k; i++) if (i != j) p *= ((m >> i) & 1) ? a1[i] : a0[i];
        s += p;
    }
    return s;
}

/* Pass 1 (Sec. III-B, Algorithm 2) and Eq. 2.  Inputs per startpoint (binary64, so that
 * finite differences can perturb them); outputs per net, declaration order:
 * sp = P(net = 1), sq = P(net = 0), tr = TR_model (startpoints: input TR when tr_mode 0). */
int orc_forward(const void *h, const double *sp_in, const double *tr_in, int tr_mode, double *sp, double *tr,
                double *sq) {
    const Orc *o = (const Orc *)h;
    for (int64_t k = 0; k < o->ns; k++) {
        int64_t n = o->start_net[k];
        sp[n] = sp_in[k];
        sq[n] = 1.0 - sp_in[k];
        tr[n] = tr_mode == 0 ? tr_in[k] : 2.0 * sp[n] * sq[n];
    }
    double a1[ORC_MAX_IN], a0[ORC_MAX_IN];
    for (int64_t t = 0; t < o->nc; t++) {
        int64_t c = o->topo[t];
        const LibCell *L = &o->lib[o->cell_lib[c]];
        for (int i = 0; i < L->k; i++) {
            int64_t f = o->fin_net[o->fin_ptr[c] + i];
            a1[i] = sp[f];
            a0[i] = sq[f];
        }
        int64_t n = o->cell_out[c];
        /* P(out=1) and P(out=0) sum to 1 in exact arithmetic; dividing by their computed
         * sum keeps rounding from accumulating along the exponentially many paths of a
         * reconvergent netlist (the sum of a cell's minterm weights is the product of its
         * fanins' sums, so any drift from 1 would otherwise add up undamped) */
        double p1 = cell_prob(L, a1, a0, 1), p0 = cell_prob(L, a1, a0, 0), s = p1 + p0;
        sp[n] = p1 / s;
        sq[n] = p0 / s;
        tr[n] = 2.0 * sp[n] * sq[n];
    }
    return 0;
}

/* Eq. 1: P = 1/2 Vdd^2 f sum_n alpha_n C_n, caps in fF.  Neumaier summation. */
double orc_power(const void *h, const double *alpha, double vdd, double fclk) {
    const Orc *o = (const Orc *)h;
    double *cl = (double *)malloc(sizeof(double) * (size_t)(o->nn + 1));
    if (!cl) return NAN;
    orc_cload(o, cl);
    double s = 0.0, comp = 0.0;
    for (int64_t n = 0; n < o->nn; n++) {
        double x = alpha[n] * cl[n];
        double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x; else comp += (x - t) + s;
        s = t;
    }
    free(cl);
    return 0.5 * vdd * vdd * fclk * 1e-15 * (s + comp);
}

/* Sec. III-E, Eq. 7 (and Eq. 6 for the hybrid modes), at the startpoint inputs sp_in/tr_in.
 *   beta      : per-net beta (NULL for grad_mode 0); the power's activity is beta * TR_model
 *               for the hybrid modes and TR_model for the model
 *   grad_mode : 0 model, 1 paper hybrid (scale accumulated gradient by beta),
 *               2 exact hybrid with beta held fixed
 * Outputs (any may be NULL): dP/d sp_in[ns], dP/d tr_in[ns], dP/d pincap[nc],
 * dP/d C_load[nn], and the full per-net SP adjoint[nn]. */
int orc_backward(const void *h, const double *sp_in, const double *tr_in, const double *beta, int grad_mode,
                 int tr_mode, double vdd, double fclk, double *g_sp_in, double *g_tr_in, double *g_pincap,
                 double *g_cload, double *g_net) {
    const Orc *o = (const Orc *)h;
    const double K = 0.5 * vdd * vdd * fclk * 1e-15;
    size_t nb = sizeof(double) * (size_t)(o->nn + 1);
    double *cl = (double *)malloc(nb), *adj = (double *)calloc((size_t)o->nn + 1, sizeof(double));
    double *tot = (double *)calloc((size_t)o->nn + 1, sizeof(double));
    double *sp = (double *)malloc(nb), *sq = (double *)malloc(nb), *tr = (double *)malloc(nb);
    if (!cl || !adj || !tot || !sp || !sq || !tr) {
        free(cl); free(adj); free(tot); free(sp); free(sq); free(tr);
        return -1;
    }
    orc_cload(o, cl);
    orc_forward(o, sp_in, tr_in, tr_mode, sp, tr, sq);
    double a1[ORC_MAX_IN], a0[ORC_MAX_IN];
    /* local term d(K C 2P(1-P))/dP = K C (2 - 4P) = 2 K C ((1-P) - P), on every net whose TR
     * comes from its SP */
    #define LOCAL(n) ((o->drv[n] >= 0 || (o->drv[n] == -1 && tr_mode == 1)) ? 2.0 * K * cl[n] * (sq[n] - sp[n]) : 0.0)
    for (int64_t t = o->nc - 1; t >= 0; t--) {
        int64_t c = o->topo[t];
        int64_t n = o->cell_out[c];
        double b = grad_mode ? beta[n] : 1.0;
        double g = grad_mode == 1 ? b * (adj[n] + LOCAL(n)) : (grad_mode == 2 ? adj[n] + b * LOCAL(n) : adj[n] + LOCAL(n));
        tot[n] = g;
        const LibCell *L = &o->lib[o->cell_lib[c]];
        for (int i = 0; i < L->k; i++) {
            int64_t f = o->fin_net[o->fin_ptr[c] + i];
            a1[i] = sp[f];
            a0[i] = sq[f];
        }
        for (int j = 0; j < L->k; j++) adj[o->fin_net[o->fin_ptr[c] + j]] += g * cell_dsp(L, a1, a0, j);
    }
    for (int64_t n = 0; n < o->nn; n++) {
        if (o->drv[n] >= 0) continue;
        double b = grad_mode ? beta[n] : 1.0;
        double l = o->drv[n] == -1 ? LOCAL(n) : 0.0;
        tot[n] = grad_mode == 1 ? b * (adj[n] + l) : (grad_mode == 2 ? adj[n] + b * l : adj[n] + l);
    }
    #undef LOCAL
    for (int64_t k = 0; k < o->ns; k++) {
        int64_t n = o->start_net[k];
        double b = grad_mode ? beta[n] : 1.0;
        if (g_sp_in) g_sp_in[k] = tot[n];
        if (g_tr_in) g_tr_in[k] = tr_mode == 0 ? K * b * cl[n] : 0.0;
    }
    #define ALPHA(n) (grad_mode ? beta[n] * tr[n] : tr[n])
    if (g_cload) for (int64_t n = 0; n < o->nn; n++) g_cload[n] = K * ALPHA(n);
    if (g_pincap)
        for (int64_t c = 0; c < o->nc; c++) {
            double s = 0.0;
            for (int64_t e = o->fin_ptr[c]; e < o->fin_ptr[c + 1]; e++) s += ALPHA(o->fin_net[e]);
            g_pincap[c] = K * s;
        }
    #undef ALPHA
    if (g_net) memcpy(g_net, tot, sizeof(double) * (size_t)o->nn);
    free(cl); free(adj); free(tot); free(sp); free(sq); free(tr);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC 2011): 10 rounds; each round multiplies the   */
/* even words by the two round constants, xors the high halves with the  */
/* odd words and the key, and the key advances by the Weyl constants.    */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* a 16-bit draw u is below the threshold with probability thr(p) / 2^16 */
static uint32_t thr(double p) {
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 65536u;
    return (uint32_t)floor(p * 65536.0);
}

static int popc64(uint64_t x) { int c = 0; while (x) { x &= x - 1; c++; } return c; }

/* Pass 2 (Sec. III-C): Markov-chain startpoint vectors, bit-packed simulation,
 * PopCount toggle counts (Eq. 4 numerator) and ones counts.
 *   words[nn * T] (may be NULL), toggles[nn], ones[nn], per net in declaration order. */
int orc_simulate(const void *h, const float *sp_in, const float *tr_in, uint64_t seed, int T,
                 uint64_t *words_out, uint32_t *toggles, uint32_t *ones) {
    const Orc *o = (const Orc *)h;
    if (T < 1) return -1;
    uint64_t *w = words_out ? words_out : (uint64_t *)malloc(sizeof(uint64_t) * (size_t)o->nn * (size_t)T + 8);
    if (!w) return -1;
    memset(w, 0, sizeof(uint64_t) * (size_t)o->nn * (size_t)T);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t k = 0; k < o->ns; k++) {
        uint64_t *wk = w + (size_t)o->start_net[k] * (size_t)T;
        double sp = (double)sp_in[k], tr = (double)tr_in[k];
        double p10 = sp > 0.0 ? tr / (2.0 * sp) : 0.0;
        double p01 = sp < 1.0 ? tr / (2.0 * (1.0 - sp)) : 0.0;
        uint32_t t_init = thr(sp), t10 = thr(p10), t01 = thr(p01);
        for (int q = 0; q < 16; q++) {
            int bit[4] = {0, 0, 0, 0};
            uint32_t u[4] = {0, 0, 0, 0};
            for (int t = 0; t < T; t++) {
                if ((t & 1) == 0) {
                    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(t / 2), (uint32_t)q, 0u};
                    orc_philox4x32_10(ctr, key, u);
                }
                for (int r = 0; r < 4; r++) {
                    uint32_t d = (t & 1) ? (u[r] >> 16) : (u[r] & 0xFFFFu);
                    if (t == 0) bit[r] = d < t_init;
                    else if (d < (bit[r] ? t10 : t01)) bit[r] ^= 1;
                    if (bit[r]) wk[t] |= 1ull << (16 * r + q);
                }
            }
        }
    }
    /* cells in topological order: out word = OR over true minterms of AND_i (x_i or ~x_i) */
    for (int64_t t0 = 0; t0 < o->nc; t0++) {
        int64_t c = o->topo[t0];
        const LibCell *L = &o->lib[o->cell_lib[c]];
        uint64_t *wo = w + (size_t)o->cell_out[c] * (size_t)T;
        int64_t M = (int64_t)1 << L->k;
        for (int t = 0; t < T; t++) {
            uint64_t acc = 0;
            for (int64_t m = 0; m < M; m++) {
                if (!L->tt[m]) continue;
                uint64_t term = ~0ull;
                for (int i = 0; i < L->k; i++) {
                    uint64_t x = w[(size_t)o->fin_net[o->fin_ptr[c] + i] * (size_t)T + (size_t)t];
                    term &= ((m >> i) & 1) ? x : ~x;
                }
                acc |= term;
            }
            wo[t] = acc;
        }
    }
    for (int64_t n = 0; n < o->nn; n++) {
        const uint64_t *wn = w + (size_t)n * (size_t)T;
        uint32_t tg = 0, on = 0;
        for (int t = 0; t < T; t++) {
            on += (uint32_t)popc64(wn[t]);
            if (t > 0) tg += (uint32_t)popc64(wn[t] ^ wn[t - 1]);
        }
        if (toggles) toggles[n] = tg;
        if (ones) ones[n] = on;
    }
    if (!words_out) free(w);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Lag-one mode (an extension of Eq. 2, Sec. II-B): every net carries   */
/* (P, T), T = P(x_t != x_{t+1}) of a stationary two-state process, so   */
/* the joint law of two consecutive values is q(1,1) = P - T/2,          */
/* q(0,0) = P(x=0) - T/2, q(0,1) = q(1,0) = T/2.  Under spatial          */
/* independence a cell toggles with probability                          */
/*   T_y = sum over input pairs (a, b) of prod_i q_i(a_i, b_i) [f(a) != f(b)], */
/* exact on fanout-free circuits; with T = 2P(1-P) at every startpoint   */
/* (temporal independence) it equals Eq. 2 on every net.                 */
/* ------------------------------------------------------------------ */

/* q(a, b) of a net, index 2a + b */
static void lag1_w(double p1, double p0, double t, double w[4]) {
    w[0] = p0 - 0.5 * t;
    w[1] = 0.5 * t;
    w[2] = 0.5 * t;
    w[3] = p1 - 0.5 * t;
}

/* sum over (a, b) of prod_i W_i[2 a_i + b_i] [f(a) != f(b)], where input `sub` (if >= 0)
 * uses the weights dsub instead of its own */
static double cell_toggle(const LibCell *L, const double (*w)[4], int sub, const double *dsub) {
    int64_t M = (int64_t)1 << L->k;
    double s = 0.0;
    for (int64_t a = 0; a < M; a++)
        for (int64_t b = 0; b < M; b++) {
            if (L->tt[a] == L->tt[b]) continue;
            double p = 1.0;
            for (int i = 0; i < L->k; i++) {
                int d = (int)(2 * ((a >> i) & 1) + ((b >> i) & 1));
                p *= i == sub ? dsub[d] : w[i][d];
            }
            s += p;
        }
    return s;
}

/* Forward of the lag-one mode: sp, sq as orc_forward; tr = T of every net. */
int orc_forward_lag1(const void *h, const double *sp_in, const double *tr_in, double *sp, double *tr, double *sq) {
    const Orc *o = (const Orc *)h;
    orc_forward(o, sp_in, tr_in, 0, sp, tr, sq);   /* SP and P(net = 0); tr is rewritten below */
    for (int64_t k = 0; k < o->ns; k++) tr[o->start_net[k]] = tr_in[k];
    double w[ORC_MAX_IN][4];
    for (int64_t t = 0; t < o->nc; t++) {
        int64_t c = o->topo[t];
        const LibCell *L = &o->lib[o->cell_lib[c]];
        for (int i = 0; i < L->k; i++) {
            int64_t f = o->fin_net[o->fin_ptr[c] + i];
            lag1_w(sp[f], sq[f], tr[f], w[i]);
        }
        tr[o->cell_out[c]] = cell_toggle(L, (const double (*)[4])w, -1, NULL);
    }
    return 0;
}

/* Gradients of P = K sum_n T_n C_n in the lag-one mode: adjoints of P and T
 * per net, in reverse topological order; outputs as orc_backward. */
int orc_backward_lag1(const void *h, const double *sp_in, const double *tr_in, double vdd, double fclk,
                      double *g_sp_in, double *g_tr_in, double *g_pincap, double *g_cload) {
    const Orc *o = (const Orc *)h;
    const double K = 0.5 * vdd * vdd * fclk * 1e-15;
    size_t nb = sizeof(double) * (size_t)(o->nn + 1);
    double *cl = (double *)malloc(nb), *sp = (double *)malloc(nb), *sq = (double *)malloc(nb);
    double *tr = (double *)malloc(nb), *gp = (double *)calloc((size_t)o->nn + 1, sizeof(double));
    double *gt = (double *)calloc((size_t)o->nn + 1, sizeof(double));
    if (!cl || !sp || !sq || !tr || !gp || !gt) {
        free(cl); free(sp); free(sq); free(tr); free(gp); free(gt);
        return -1;
    }
    orc_cload(o, cl);
    orc_forward_lag1(o, sp_in, tr_in, sp, tr, sq);
    for (int64_t n = 0; n < o->nn; n++) gt[n] = K * cl[n];   /* dP/dT_n, direct */
    static const double dP[4] = {-1.0, 0.0, 0.0, 1.0};       /* d q(a,b) / dP */
    static const double dT[4] = {-0.5, 0.5, 0.5, -0.5};      /* d q(a,b) / dT */
    double w[ORC_MAX_IN][4], a1[ORC_MAX_IN], a0[ORC_MAX_IN];
    for (int64_t t = o->nc - 1; t >= 0; t--) {
        int64_t c = o->topo[t];
        int64_t y = o->cell_out[c];
        const LibCell *L = &o->lib[o->cell_lib[c]];
        for (int i = 0; i < L->k; i++) {
            int64_t f = o->fin_net[o->fin_ptr[c] + i];
            lag1_w(sp[f], sq[f], tr[f], w[i]);
            a1[i] = sp[f];
            a0[i] = sq[f];
        }
        for (int i = 0; i < L->k; i++) {
            int64_t f = o->fin_net[o->fin_ptr[c] + i];
            double dty_dp = cell_toggle(L, (const double (*)[4])w, i, dP);
            double dty_dt = cell_toggle(L, (const double (*)[4])w, i, dT);
            gp[f] += gp[y] * cell_dsp(L, a1, a0, i) + gt[y] * dty_dp;
            gt[f] += gt[y] * dty_dt;
        }
    }
    for (int64_t k = 0; k < o->ns; k++) {
        int64_t n = o->start_net[k];
        if (g_sp_in) g_sp_in[k] = gp[n];
        if (g_tr_in) g_tr_in[k] = gt[n];
    }
    if (g_cload) for (int64_t n = 0; n < o->nn; n++) g_cload[n] = K * tr[n];
    if (g_pincap)
        for (int64_t c = 0; c < o->nc; c++) {
            double s = 0.0;
            for (int64_t e = o->fin_ptr[c]; e < o->fin_ptr[c + 1]; e++) s += tr[o->fin_net[e]];
            g_pincap[c] = K * s;
        }
    free(cl); free(sp); free(sq); free(tr); free(gp); free(gt);
    return 0;
}

/* Logic values of every net for 64 input vectors at once (Eq. 3 needs val_i(v)):
 * bit b of start_words[k] is the value of startpoint k in vector b; each cell, in
 * topological order, ORs the AND-terms of its true minterms over its input words.
 * net_words[nn] in declaration order. */
void orc_logic_words(const void *h, const uint64_t *start_words, uint64_t *net_words) {
    const Orc *o = (const Orc *)h;
    for (int64_t n = 0; n < o->nn; n++) net_words[n] = 0;
    for (int64_t k = 0; k < o->ns; k++) net_words[o->start_net[k]] = start_words[k];
    for (int64_t t0 = 0; t0 < o->nc; t0++) {
        int64_t c = o->topo[t0];
        const LibCell *L = &o->lib[o->cell_lib[c]];
        int64_t M = (int64_t)1 << L->k;
        uint64_t acc = 0;
        for (int64_t m = 0; m < M; m++) {
            if (!L->tt[m]) continue;
            uint64_t term = ~0ull;
            for (int i = 0; i < L->k; i++) {
                uint64_t x = net_words[o->fin_net[o->fin_ptr[c] + i]];
                term &= ((m >> i) & 1) ? x : ~x;
            }
            acc |= term;
        }
        net_words[o->cell_out[c]] = acc;
    }
}

/* Sec. III-D, Eq. 4 and Eq. 5: TR_acc = toggles / (64 (T-1)), beta = clip(TR_acc / TR_model),
 * hybrid activity = beta * TR_model. */
void orc_hybrid(const void *h, const double *tr_model, const uint32_t *toggles, int T, double beta_min,
                double beta_max, double *beta, double *tr_hyb) {
    const Orc *o = (const Orc *)h;
    double nsim = 64.0 * (double)(T > 1 ? T - 1 : 1);
    for (int64_t n = 0; n < o->nn; n++) {
        double acc = (double)toggles[n] / nsim;
        double b;
        if (tr_model[n] > 0.0) {
            b = acc / tr_model[n];
            if (b < beta_min) b = beta_min;
            if (b > beta_max) b = beta_max;
        } else {
            b = acc == 0.0 ? 1.0 : beta_max;
        }
        beta[n] = b;
        tr_hyb[n] = b * tr_model[n];
    }
}


/* ------------------------------------------------------------------ */
/* Level-parallel variants (OpenMP) for the CPU baseline of the        */
/* benchmark: the same per-cell arithmetic as orc_forward, orc_simulate */
/* and orc_backward, with the cells of one level processed in parallel  */
/* (all fanins of a cell lie on lower levels).  The forward pass and   */
/* the simulation give bitwise the same results as the serial ones;    */
/* the adjoint gathers each net's contributions over its sinks instead  */
/* of scattering them, so it agrees to rounding.                       */
/* ------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void par_fwd_cell(const Orc *o, int64_t c, double *sp, double *tr, double *sq) {
    const LibCell *L = &o->lib[o->cell_lib[c]];
    double a1[ORC_MAX_IN], a0[ORC_MAX_IN];
    for (int i = 0; i < L->k; i++) {
        int64_t f = o->fin_net[o->fin_ptr[c] + i];
        a1[i] = sp[f];
        a0[i] = sq[f];
    }
    int64_t n = o->cell_out[c];
    double p1 = cell_prob(L, a1, a0, 1), p0 = cell_prob(L, a1, a0, 0), s = p1 + p0;
    sp[n] = p1 / s;
    sq[n] = p0 / s;
    tr[n] = 2.0 * sp[n] * sq[n];
}

int orc_forward_par(const void *h, const double *sp_in, const double *tr_in, int tr_mode, double *sp, double *tr,
                    double *sq) {
    const Orc *o = (const Orc *)h;
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < o->ns; k++) {
        int64_t n = o->start_net[k];
        sp[n] = sp_in[k];
        sq[n] = 1.0 - sp_in[k];
        tr[n] = tr_mode == 0 ? tr_in[k] : 2.0 * sp[n] * sq[n];
    }
    for (int32_t l = 1; l <= o->depth; l++) {
        const int64_t i0 = o->lvl_ptr[l - 1], i1 = o->lvl_ptr[l];
        #pragma omp parallel for schedule(static)
        for (int64_t i = i0; i < i1; i++) par_fwd_cell(o, o->lvl_cell[i], sp, tr, sq);
    }
    return 0;
}

/* the Markov chains of startpoint k (the serial simulation's startpoint loop body) */
static void par_sim_start(const Orc *o, int64_t k, const float *sp_in, const float *tr_in, const uint32_t key[2],
                          int T, uint64_t *w) {
    uint64_t *wk = w + (size_t)o->start_net[k] * (size_t)T;
    double sp = (double)sp_in[k], tr = (double)tr_in[k];
    double p10 = sp > 0.0 ? tr / (2.0 * sp) : 0.0;
    double p01 = sp < 1.0 ? tr / (2.0 * (1.0 - sp)) : 0.0;
    uint32_t t_init = thr(sp), t10 = thr(p10), t01 = thr(p01);
    for (int q = 0; q < 16; q++) {
        int bit[4] = {0, 0, 0, 0};
        uint32_t u[4] = {0, 0, 0, 0};
        for (int t = 0; t < T; t++) {
            if ((t & 1) == 0) {
                uint32_t ctr[4] = {(uint32_t)k, (uint32_t)(t / 2), (uint32_t)q, 0u};
                orc_philox4x32_10(ctr, key, u);
            }
            for (int r = 0; r < 4; r++) {
                uint32_t d = (t & 1) ? (u[r] >> 16) : (u[r] & 0xFFFFu);
                if (t == 0) bit[r] = d < t_init;
                else if (d < (bit[r] ? t10 : t01)) bit[r] ^= 1;
                if (bit[r]) wk[t] |= 1ull << (16 * r + q);
            }
        }
    }
}

static void par_sim_cell(const Orc *o, int64_t c, int T, uint64_t *w) {
    const LibCell *L = &o->lib[o->cell_lib[c]];
    uint64_t *wo = w + (size_t)o->cell_out[c] * (size_t)T;
    int64_t M = (int64_t)1 << L->k;
    for (int t = 0; t < T; t++) {
        uint64_t acc = 0;
        for (int64_t m = 0; m < M; m++) {
            if (!L->tt[m]) continue;
            uint64_t term = ~0ull;
            for (int i = 0; i < L->k; i++) {
                uint64_t x = w[(size_t)o->fin_net[o->fin_ptr[c] + i] * (size_t)T + (size_t)t];
                term &= ((m >> i) & 1) ? x : ~x;
            }
            acc |= term;
        }
        wo[t] = acc;
    }
}

int orc_simulate_par(const void *h, const float *sp_in, const float *tr_in, uint64_t seed, int T,
                     uint64_t *words_out, uint32_t *toggles, uint32_t *ones) {
    const Orc *o = (const Orc *)h;
    if (T < 1) return -1;
    uint64_t *w = words_out ? words_out : (uint64_t *)malloc(sizeof(uint64_t) * (size_t)o->nn * (size_t)T + 8);
    if (!w) return -1;
    memset(w, 0, sizeof(uint64_t) * (size_t)o->nn * (size_t)T);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < o->ns; k++) par_sim_start(o, k, sp_in, tr_in, key, T, w);
    for (int32_t l = 1; l <= o->depth; l++) {
        const int64_t i0 = o->lvl_ptr[l - 1], i1 = o->lvl_ptr[l];
        #pragma omp parallel for schedule(static)
        for (int64_t i = i0; i < i1; i++) par_sim_cell(o, o->lvl_cell[i], T, w);
    }
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < o->nn; n++) {
        const uint64_t *wn = w + (size_t)n * (size_t)T;
        uint32_t tg = 0, on = 0;
        for (int t = 0; t < T; t++) {
            on += (uint32_t)popc64(wn[t]);
            if (t > 0) tg += (uint32_t)popc64(wn[t] ^ wn[t - 1]);
        }
        if (toggles) toggles[n] = tg;
        if (ones) ones[n] = on;
    }
    if (!words_out) free(w);
    return 0;
}

/* sum over the sink pins (c, j) of net n of tot[out(c)] * d SP_out(c) / d a_j */
static double par_sink_sum(const Orc *o, int64_t n, const double *tot, const double *sp, const double *sq) {
    double s = 0.0;
    int64_t prev = -1;
    double a1[ORC_MAX_IN], a0[ORC_MAX_IN];
    for (int64_t e = o->sink_ptr[n]; e < o->sink_ptr[n + 1]; e++) {
        int64_t c = o->sink_cell[e];
        if (c == prev) continue;   /* a cell reading n on several pins is listed once per pin */
        prev = c;
        const LibCell *L = &o->lib[o->cell_lib[c]];
        for (int i = 0; i < L->k; i++) {
            int64_t f = o->fin_net[o->fin_ptr[c] + i];
            a1[i] = sp[f];
            a0[i] = sq[f];
        }
        for (int j = 0; j < L->k; j++)
            if (o->fin_net[o->fin_ptr[c] + j] == n) s += tot[o->cell_out[c]] * cell_dsp(L, a1, a0, j);
    }
    return s;
}

int orc_backward_par(const void *h, const double *sp_in, const double *tr_in, const double *beta, int grad_mode,
                     int tr_mode, double vdd, double fclk, double *g_sp_in, double *g_tr_in, double *g_pincap,
                     double *g_cload, double *g_net) {
    const Orc *o = (const Orc *)h;
    const double K = 0.5 * vdd * vdd * fclk * 1e-15;
    size_t nb = sizeof(double) * (size_t)(o->nn + 1);
    double *cl = (double *)malloc(nb), *tot = (double *)calloc((size_t)o->nn + 1, sizeof(double));
    double *sp = (double *)malloc(nb), *sq = (double *)malloc(nb), *tr = (double *)malloc(nb);
    if (!cl || !tot || !sp || !sq || !tr) {
        free(cl); free(tot); free(sp); free(sq); free(tr);
        return -1;
    }
    orc_cload(o, cl);
    orc_forward_par(o, sp_in, tr_in, tr_mode, sp, tr, sq);
    #define LOCAL(n) ((o->drv[n] >= 0 || (o->drv[n] == -1 && tr_mode == 1)) ? 2.0 * K * cl[n] * (sq[n] - sp[n]) : 0.0)
    #define COMBINE(acc, l, b) (grad_mode == 1 ? (b) * ((acc) + (l)) : (grad_mode == 2 ? (acc) + (b) * (l) : (acc) + (l)))
    for (int32_t l = o->depth; l >= 1; l--) {
        const int64_t i0 = o->lvl_ptr[l - 1], i1 = o->lvl_ptr[l];
        #pragma omp parallel for schedule(static)
        for (int64_t i = i0; i < i1; i++) {
            int64_t n = o->cell_out[o->lvl_cell[i]];
            double b = grad_mode ? beta[n] : 1.0;
            tot[n] = COMBINE(par_sink_sum(o, n, tot, sp, sq), LOCAL(n), b);
        }
    }
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < o->ns; k++) {
        int64_t n = o->start_net[k];
        double b = grad_mode ? beta[n] : 1.0;
        tot[n] = COMBINE(par_sink_sum(o, n, tot, sp, sq), LOCAL(n), b);
    }
    #undef COMBINE
    #undef LOCAL
    for (int64_t k = 0; k < o->ns; k++) {
        int64_t n = o->start_net[k];
        double b = grad_mode ? beta[n] : 1.0;
        if (g_sp_in) g_sp_in[k] = tot[n];
        if (g_tr_in) g_tr_in[k] = tr_mode == 0 ? K * b * cl[n] : 0.0;
    }
    #define ALPHA(n) (grad_mode ? beta[n] * tr[n] : tr[n])
    if (g_cload) {
        #pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < o->nn; n++) g_cload[n] = K * ALPHA(n);
    }
    if (g_pincap) {
        #pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < o->nc; c++) {
            double s = 0.0;
            for (int64_t e = o->fin_ptr[c]; e < o->fin_ptr[c + 1]; e++) s += ALPHA(o->fin_net[e]);
            g_pincap[c] = K * s;
        }
    }
    #undef ALPHA
    if (g_net) memcpy(g_net, tot, sizeof(double) * (size_t)o->nn);
    free(cl); free(tot); free(sp); free(sq); free(tr);
    return 0;
}
