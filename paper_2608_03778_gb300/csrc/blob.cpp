// Compiled netlists as byte blobs (the "compiled bytecode netlist" form of the
// design, Sec. III-A, Algorithm 1): compile once on any host, store the blob,
// load it later without the netlist text.
//
// Layout (little-endian, as both supported hosts are): the 8-byte tag
// "DPBLOB01", six int64 sizes (nets, startpoints, cells, edges, levels, logic
// ids in use), then each array as an int64 element count followed by its
// elements, in a fixed order.  Loading checks every size and every value the
// device kernels rely on - level bounds, fanin ids below the cell's own level,
// the fanout CSR and edge positions against the fanin records, the two
// permutations, finite non-negative caps, the bytecode ranges - so a damaged
// blob is rejected with DP_EPARSE instead of reaching the GPU.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "compiled.h"

namespace {

constexpr char kTag[8] = {'D', 'P', 'B', 'L', 'O', 'B', '0', '1'};

struct Writer {
    unsigned char *buf;
    size_t cap, len = 0;
    void raw(const void *p, size_t n) {
        if (buf && len + n <= cap) std::memcpy(buf + len, p, n);
        len += n;
    }
    void i64(int64_t v) { raw(&v, sizeof v); }
    template <class T>
    void arr(const T *p, size_t n) {
        i64((int64_t)n);
        raw(p, sizeof(T) * n);
    }
    template <class T>
    void vec(const std::vector<T> &v) {
        arr(v.data(), v.size());
    }
};

struct Reader {
    const unsigned char *p;
    size_t len, at = 0;
    bool ok = true;
    bool raw(void *dst, size_t n) {
        if (!ok || n > len - at) return ok = false;
        std::memcpy(dst, p + at, n);
        at += n;
        return true;
    }
    int64_t i64() {
        int64_t v = 0;
        raw(&v, sizeof v);
        return v;
    }
    // an array of exactly `want` elements
    template <class T>
    bool vec(std::vector<T> *v, int64_t want) {
        const int64_t n = i64();
        if (!ok || n != want || want < 0 || (uint64_t)want > (len - at) / sizeof(T)) return ok = false;
        v->resize((size_t)want);
        return raw(v->data(), sizeof(T) * (size_t)want);
    }
    template <class T>
    bool fixed(T *dst, int64_t want) {
        const int64_t n = i64();
        if (!ok || n != want) return ok = false;
        return raw(dst, sizeof(T) * (size_t)want);
    }
};

bool is_permutation(const std::vector<int32_t> &a) {
    std::vector<char> seen(a.size(), 0);
    for (int32_t x : a) {
        if (x < 0 || (size_t)x >= a.size() || seen[(size_t)x]) return false;
        seen[(size_t)x] = 1;
    }
    return true;
}

// every structural property the device code assumes; the first one violated, or "" if none
std::string check(const dp_compiled &c) {
    const int64_t nn = c.n_nets, ns = c.n_start, nc = c.n_cells, ne = c.n_edges;
    const int L = c.n_levels;
    if (ns < 0 || nc < 0 || ne < 0 || L < 0 || nn != ns + nc || nn > dp::kMaxNets) return "sizes";
    if (c.lvl_ptr.empty() || c.lvl_ptr[0] != 0 || c.lvl_ptr[(size_t)L] != nc) return "level bounds";
    for (int l = 1; l <= L; l++)
        if (c.lvl_ptr[(size_t)l] < c.lvl_ptr[(size_t)l - 1]) return "level bounds";
    for (int i = 0; i < 256; i++)
        if (c.op_arity[i] > dp::kMaxArity) return "logic arity";
    // level of every net: startpoints 0, cell i's net its level
    std::vector<int32_t> lvl_of((size_t)nn, 0);
    for (int l = 1; l <= L; l++)
        for (int32_t i = c.lvl_ptr[(size_t)l - 1]; i < c.lvl_ptr[(size_t)l]; i++) lvl_of[(size_t)(ns + i)] = l;
    std::vector<int32_t> fanout_count((size_t)nn, 0);
    for (int l = 1; l <= L; l++)
        for (int32_t i = c.lvl_ptr[(size_t)l - 1]; i < c.lvl_ptr[(size_t)l]; i++) {
            const uint32_t *r = &c.fanin[4 * (size_t)i];
            const int k = c.op_arity[r[0] >> 24];
            for (int j = 0; j < 4; j++) {
                const uint32_t n = j == 0 ? (r[0] & dp::kNetMask) : r[j];
                if (j >= k) {
                    if (c.edge_fpos[4 * (size_t)i + j] != -1) return "unused fanin slot";
                    continue;
                }
                if ((int64_t)n >= nn || lvl_of[n] >= l) return "fanin below the cell's level";
                fanout_count[n]++;
            }
        }
    if (c.fout_ptr[0] != 0 || c.fout_ptr[(size_t)nn] != ne) return "fanout bounds";
    for (int64_t n = 0; n < nn; n++) {
        if (c.fout_ptr[(size_t)n + 1] - c.fout_ptr[(size_t)n] != fanout_count[(size_t)n]) return "fanout counts";
        for (int32_t e = c.fout_ptr[(size_t)n]; e < c.fout_ptr[(size_t)n + 1]; e++) {
            const int32_t edge = c.fout_edge[(size_t)e];
            if (edge < 0 || edge / 4 >= nc) return "fanout edge";
            const int32_t cell = edge / 4, slot = edge % 4;
            const uint32_t *r = &c.fanin[4 * (size_t)cell];
            const uint32_t src = slot == 0 ? (r[0] & dp::kNetMask) : r[slot];
            if (slot >= c.op_arity[r[0] >> 24] || (int64_t)src != n) return "fanout edge";
            if (c.edge_fpos[(size_t)edge] != e) return "edge position";
        }
    }
    if (!is_permutation(c.net_of_user) || !is_permutation(c.user_of_net) || !is_permutation(c.cell_of_user) ||
        !is_permutation(c.user_of_cell))
        return "user order";
    for (int64_t n = 0; n < nn; n++)
        if (c.user_of_net[(size_t)c.net_of_user[(size_t)n]] != n) return "user order";
    for (int64_t i = 0; i < nc; i++)
        if (c.user_of_cell[(size_t)c.cell_of_user[(size_t)i]] != i) return "user order";
    for (float x : c.base_cap)
        if (!(x >= 0.f) || !std::isfinite(x)) return "caps";
    for (float x : c.pincap)
        if (!(x >= 0.f) || !std::isfinite(x)) return "caps";
    const int64_t nbc = (int64_t)c.bc_ops.size();
    for (int i = 0; i < 256; i++)
        if (c.bc_offset[i] < -1 || c.bc_length[i] < 0 || (c.bc_offset[i] >= 0 && c.bc_offset[i] + (int64_t)c.bc_length[i] > nbc))
            return "bytecode ranges";
    return "";
}

}  // namespace

extern "C" dp_status dp_compiled_save(const dp_compiled *c, void *buf, size_t cap, size_t *len) {
    if (!c || !len) return DP_EINVAL;
    Writer w{static_cast<unsigned char *>(buf), cap};
    w.raw(kTag, sizeof kTag);
    for (int64_t v : {c->n_nets, c->n_start, c->n_cells, c->n_edges, (int64_t)c->n_levels, (int64_t)c->n_ops})
        w.i64(v);
    w.vec(c->lvl_ptr);
    w.vec(c->fanin);
    w.vec(c->fout_ptr);
    w.vec(c->fout_edge);
    w.vec(c->edge_fpos);
    w.vec(c->net_of_user);
    w.vec(c->user_of_net);
    w.vec(c->cell_of_user);
    w.vec(c->user_of_cell);
    w.vec(c->base_cap);
    w.vec(c->pincap);
    w.arr(c->op_arity, 256);
    w.arr(c->op_tt, 256);
    w.vec(c->bc_ops);
    w.vec(c->bc_args);
    w.arr(c->bc_offset, 256);
    w.arr(c->bc_length, 256);
    *len = w.len;
    if (buf && cap < w.len) return DP_EINVAL;
    return DP_OK;
}

extern "C" dp_status dp_compiled_load(const void *blob, size_t len, dp_compiled **out, char *errbuf, size_t errlen) {
    auto fail = [&](dp_status s, const char *what) {
        if (errbuf && errlen) std::snprintf(errbuf, errlen, "compiled blob: %s", what);
        return s;
    };
    if (!out || (!blob && len)) return fail(DP_EINVAL, "NULL argument");
    *out = nullptr;
    Reader r{static_cast<const unsigned char *>(blob), len};
    char tag[8] = {0};
    if (!r.raw(tag, sizeof tag) || std::memcmp(tag, kTag, sizeof kTag) != 0) return fail(DP_EPARSE, "not a blob");
    dp_compiled *c = new (std::nothrow) dp_compiled();
    if (!c) return fail(DP_ENOMEM, "out of memory");
    c->n_nets = r.i64();
    c->n_start = r.i64();
    c->n_cells = r.i64();
    c->n_edges = r.i64();
    const int64_t L = r.i64(), nops = r.i64();
    const int64_t nn = c->n_nets, nc = c->n_cells, ne = c->n_edges;
    bool ok = r.ok && nn >= 0 && nc >= 0 && ne >= 0 && L >= 0 && nn <= dp::kMaxNets && nc <= nn && L <= nc + 1 &&
              nops >= 0 && nops <= 256 && ne <= 4 * nc;
    if (ok) {
        c->n_levels = (int32_t)L;
        c->n_ops = (int32_t)nops;
        try {
            ok = r.vec(&c->lvl_ptr, L + 1) && r.vec(&c->fanin, 4 * nc) && r.vec(&c->fout_ptr, nn + 1) &&
                 r.vec(&c->fout_edge, ne) && r.vec(&c->edge_fpos, 4 * nc) && r.vec(&c->net_of_user, nn) &&
                 r.vec(&c->user_of_net, nn) && r.vec(&c->cell_of_user, nc) && r.vec(&c->user_of_cell, nc) &&
                 r.vec(&c->base_cap, nn) && r.vec(&c->pincap, nc) && r.fixed(c->op_arity, 256) &&
                 r.fixed(c->op_tt, 256);
            if (ok) {
                const int64_t nbc = r.i64();
                ok = r.ok && nbc >= 0 && (uint64_t)nbc <= len - r.at;
                r.at -= sizeof(int64_t);   // re-read as the vector's own count
                ok = ok && r.vec(&c->bc_ops, nbc) && r.vec(&c->bc_args, nbc) && r.fixed(c->bc_offset, 256) &&
                     r.fixed(c->bc_length, 256) && r.at == len;
            }
        } catch (const std::bad_alloc &) {
            delete c;
            return fail(DP_ENOMEM, "out of memory");
        }
    }
    if (!ok) {
        delete c;
        return fail(DP_EPARSE, "truncated or inconsistent sizes");
    }
    const std::string bad = check(*c);
    if (!bad.empty()) {
        delete c;
        return fail(DP_EPARSE, bad.c_str());
    }
    *out = c;
    return DP_OK;
}
