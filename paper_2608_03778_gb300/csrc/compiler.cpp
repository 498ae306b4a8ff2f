// Host compiler: library functions -> bytecode -> truth tables (Sec. III-A,
// Algorithm 1), netlist -> levelized, opcode-sorted fanin records and the
// transposed fanout CSR used by the GPU kernels.
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <string_view>
#include <unordered_map>
#include <vector>

#include "compiled.h"

namespace dp {
namespace {

// ---------------------------------------------------------------- lexer ----
enum Tok { T_ID, T_AND, T_OR, T_XOR, T_NOT, T_POSTNOT, T_LP, T_RP, T_C0, T_C1, T_END, T_BAD };
struct Token { Tok t; std::string s; };

std::vector<Token> lex(const std::string &e) {
    std::vector<Token> out;
    size_t i = 0;
    while (i < e.size()) {
        char c = e[i];
        if (c == ' ' || c == '\t' || c == '\r') { i++; continue; }
        if (std::isalpha((unsigned char)c) || c == '_') {
            size_t j = i;
            while (j < e.size() && (std::isalnum((unsigned char)e[j]) || e[j] == '_')) j++;
            out.push_back({T_ID, e.substr(i, j - i)});
            i = j;
            continue;
        }
        Tok t = T_BAD;
        switch (c) {
            case '&': case '*': t = T_AND; break;
            case '|': case '+': t = T_OR; break;
            case '^': t = T_XOR; break;
            case '!': case '~': t = T_NOT; break;
            case '\'': t = T_POSTNOT; break;
            case '(': t = T_LP; break;
            case ')': t = T_RP; break;
            case '0': t = T_C0; break;
            case '1': t = T_C1; break;
            default: break;
        }
        out.push_back({t, std::string(1, c)});
        i++;
    }
    out.push_back({T_END, ""});
    return out;
}

// --------------------------------------------------------------- parser ----
// AST nodes in a flat vector; precedence NOT > AND > XOR > OR.
struct Node { BcOp op; int a = -1, b = -1; std::string name; };

struct Parser {
    const std::vector<Token> &tk;
    size_t p = 0;
    std::vector<Node> nodes;
    std::string err;
    explicit Parser(const std::vector<Token> &t) : tk(t) {}
    int mk(Node n) { nodes.push_back(std::move(n)); return (int)nodes.size() - 1; }
    int primary() {
        const Token &t = tk[p];
        if (t.t == T_LP) {
            p++;
            int v = orx();
            if (v < 0) return -1;
            if (tk[p].t != T_RP) { err = "missing ')'"; return -1; }
            p++;
            return v;
        }
        if (t.t == T_ID) { p++; Node n{BC_IN}; n.name = t.s; return mk(n); }
        if (t.t == T_C0 || t.t == T_C1) { p++; return mk(Node{t.t == T_C1 ? BC_C1 : BC_C0}); }
        err = "unexpected '" + t.s + "'";
        return -1;
    }
    int unary() {
        if (tk[p].t == T_NOT) {
            p++;
            int v = unary();
            if (v < 0) return -1;
            Node n{BC_NOT}; n.a = v; return mk(n);
        }
        int v = primary();
        while (v >= 0 && tk[p].t == T_POSTNOT) { p++; Node n{BC_NOT}; n.a = v; v = mk(n); }
        return v;
    }
    int binary(int level) {
        static const Tok tok_of[3] = {T_OR, T_XOR, T_AND};
        static const BcOp op_of[3] = {BC_OR, BC_XOR, BC_AND};
        int v = level == 3 ? unary() : binary(level + 1);
        if (level == 3) return v;
        while (v >= 0 && tk[p].t == tok_of[level]) {
            p++;
            int w = binary(level + 1);
            if (w < 0) return -1;
            Node n{op_of[level]}; n.a = v; n.b = w; v = mk(n);
        }
        return v;
    }
    int orx() { return binary(0); }
};

void collect_inputs(const std::vector<Node> &nd, int i, std::vector<std::string> *order) {
    const Node &n = nd[i];
    if (n.op == BC_IN) {
        if (std::find(order->begin(), order->end(), n.name) == order->end()) order->push_back(n.name);
        return;
    }
    if (n.a >= 0) collect_inputs(nd, n.a, order);
    if (n.b >= 0) collect_inputs(nd, n.b, order);
}

void emit(const std::vector<Node> &nd, int i, const std::vector<std::string> &order, Function *f) {
    const Node &n = nd[i];
    if (n.a >= 0) emit(nd, n.a, order, f);
    if (n.b >= 0) emit(nd, n.b, order, f);
    int8_t arg = 0;
    if (n.op == BC_IN) arg = (int8_t)(std::find(order.begin(), order.end(), n.name) - order.begin());
    f->ops.push_back(n.op);
    f->args.push_back(arg);
}

// Common gates get fixed ids: BUF 0, INV 1, and for n = 2..4 inputs
// AND 2+5(n-2), OR +1, NAND +2, NOR +3, XOR +4 (left-associated chains).
int match_known(const Function &f) {
    const auto &o = f.ops;
    const auto &a = f.args;
    const int n = (int)f.inputs.size();
    if (n == 1 && o.size() == 1 && o[0] == BC_IN) return 0;
    if (n == 1 && o.size() == 2 && o[0] == BC_IN && o[1] == BC_NOT) return 1;
    if (n < 2 || n > 4) return -1;
    // IN0 IN1 X IN2 X ... [NOT]
    size_t len = 2 * (size_t)n - 1;
    bool neg = o.size() == len + 1 && o.back() == BC_NOT;
    if (o.size() != len && !neg) return -1;
    if (o[0] != BC_IN || a[0] != 0 || o[1] != BC_IN || a[1] != 1) return -1;
    BcOp x = (BcOp)o[2];
    if (x != BC_AND && x != BC_OR && x != BC_XOR) return -1;
    for (int k = 2; k < n; k++)
        if (o[2 * k - 1] != BC_IN || a[2 * k - 1] != k || o[2 * k] != x) return -1;
    int base = 2 + 5 * (n - 2);
    if (x == BC_AND) return base + (neg ? 2 : 0);
    if (x == BC_OR) return base + (neg ? 3 : 1);
    return neg ? -1 : base + 4;
}

// Runs the bytecode on Boolean inputs (bit j of m = input j).
bool run_bool(const Function &f, uint32_t m) {
    bool st[64];
    int sp = 0;
    for (size_t i = 0; i < f.ops.size(); i++) {
        switch (f.ops[i]) {
            case BC_IN: st[sp++] = (m >> f.args[i]) & 1; break;
            case BC_C0: st[sp++] = false; break;
            case BC_C1: st[sp++] = true; break;
            case BC_NOT: st[sp - 1] = !st[sp - 1]; break;
            case BC_AND: sp--; st[sp - 1] = st[sp - 1] && st[sp]; break;
            case BC_OR: sp--; st[sp - 1] = st[sp - 1] || st[sp]; break;
            case BC_XOR: sp--; st[sp - 1] = st[sp - 1] != st[sp]; break;
        }
    }
    return st[0];
}

}  // namespace

bool compile_function(const std::string &expr, Function *f, std::string *err) {
    *f = Function();
    auto tk = lex(expr);
    for (auto &t : tk)
        if (t.t == T_BAD) { *err = "bad character '" + t.s + "'"; return false; }
    Parser ps(tk);
    int root = ps.orx();
    if (root < 0) { *err = ps.err; return false; }
    if (tk[ps.p].t != T_END) { *err = "trailing '" + tk[ps.p].s + "'"; return false; }
    collect_inputs(ps.nodes, root, &f->inputs);
    if (f->inputs.size() > 16) { *err = "too many inputs"; return false; }
    emit(ps.nodes, root, f->inputs, f);
    // the stack depth of a post-order expression is bounded by its node count
    if (f->ops.size() > 60) { *err = "expression too long"; return false; }
    f->logic_id = match_known(*f);
    if (f->inputs.size() <= (size_t)kMaxArity) {
        uint16_t tt = 0;
        for (uint32_t m = 0; m < (1u << f->inputs.size()); m++)
            if (run_bool(*f, m)) tt |= (uint16_t)(1u << m);
        f->tt = tt;
    }
    return true;
}

}  // namespace dp

// ------------------------------------------------------------ netlist ------
namespace {

using dp::Function;

struct LibEntry {
    bool seq = false;
    std::string out, dpin;
    float pincap = 0;
    int op = -1;
    std::vector<std::string> pins;  // slot order
};

struct Err {
    std::string msg;
    dp_status code = DP_OK;
    bool set(dp_status c, const std::string &m, long line = -1) {
        code = c;
        msg = line >= 0 ? m + " (line " + std::to_string(line) + ")" : m;
        return false;
    }
};

// whitespace tokenizer over one line
int split(std::string_view line, std::string_view *tok, int maxtok, std::string_view *rest_after) {
    int n = 0;
    size_t i = 0;
    if (rest_after) *rest_after = std::string_view();
    while (i < line.size() && n < maxtok) {
        while (i < line.size() && (line[i] == ' ' || line[i] == '\t' || line[i] == '\r')) i++;
        if (i >= line.size()) break;
        size_t j = i;
        while (j < line.size() && line[j] != ' ' && line[j] != '\t' && line[j] != '\r') j++;
        tok[n++] = line.substr(i, j - i);
        i = j;
    }
    if (rest_after) {
        while (i < line.size() && (line[i] == ' ' || line[i] == '\t')) i++;
        size_t e = line.size();
        while (e > i && (line[e - 1] == ' ' || line[e - 1] == '\t' || line[e - 1] == '\r')) e--;
        *rest_after = line.substr(i, e - i);
    }
    return n;
}

template <class F>
void for_lines(std::string_view text, F &&f) {
    size_t pos = 0;
    long ln = 0;
    while (pos < text.size()) {
        size_t e = text.find('\n', pos);
        if (e == std::string_view::npos) e = text.size();
        std::string_view line = text.substr(pos, e - pos);
        size_t h = line.find('#');
        if (h != std::string_view::npos) line = line.substr(0, h);
        ln++;
        if (!f(line, ln)) return;
        pos = e + 1;
    }
}

bool parse_float(std::string_view s, float *out) {
    std::string t(s);
    char *end = nullptr;
    double v = std::strtod(t.c_str(), &end);
    if (end == t.c_str() || *end) return false;
    *out = (float)v;
    return true;
}

bool parse_library(std::string_view text, std::unordered_map<std::string, LibEntry> *lib, dp_compiled *c,
                   Err *err) {
    std::vector<std::pair<std::vector<uint8_t>, std::vector<int8_t>>> gen_sig;  // signature per generated id
    int next_id = dp::kGenStart;
    bool ok = true;
    for_lines(text, [&](std::string_view line, long ln) {
        std::string_view tok[5], rest;
        int n = split(line, tok, 4, &rest);
        if (n == 0 || tok[0] == "library") return true;
        LibEntry e;
        std::string name;
        if (tok[0] == "seq") {
            std::string_view t5[5];
            int m = split(line, t5, 5, nullptr);
            if (m != 5 || !parse_float(t5[4], &e.pincap)) return ok = err->set(DP_EPARSE, "bad seq line", ln);
            e.seq = true;
            name = std::string(t5[1]);
            e.dpin = std::string(t5[2]);
            e.out = std::string(t5[3]);
        } else if (tok[0] == "cell") {
            if (n < 4 || rest.empty()) return ok = err->set(DP_EPARSE, "bad cell line", ln);
            name = std::string(tok[1]);
            e.out = std::string(tok[2]);
            if (!parse_float(tok[3], &e.pincap)) return ok = err->set(DP_EPARSE, "bad pin cap", ln);
            Function f;
            std::string msg;
            if (!dp::compile_function(std::string(rest), &f, &msg))
                return ok = err->set(DP_EPARSE, "function of " + name + ": " + msg, ln);
            if ((int)f.inputs.size() > dp::kMaxArity)
                return ok = err->set(DP_EUNSUPPORTED, "cell " + name + " has more than 4 inputs", ln);
            e.pins = f.inputs;
            int id = f.logic_id;
            if (id < 0) {
                for (size_t g = 0; g < gen_sig.size() && id < 0; g++)
                    if (gen_sig[g].first == f.ops && gen_sig[g].second == f.args) id = dp::kGenStart + (int)g;
                if (id < 0) {
                    if (next_id > 255) return ok = err->set(DP_EUNSUPPORTED, "more than 224 distinct functions", ln);
                    id = next_id++;
                    gen_sig.push_back({f.ops, f.args});
                    c->bc_offset[id] = (int32_t)c->bc_ops.size();
                    c->bc_length[id] = (int32_t)f.ops.size();
                    c->bc_ops.insert(c->bc_ops.end(), f.ops.begin(), f.ops.end());
                    c->bc_args.insert(c->bc_args.end(), f.args.begin(), f.args.end());
                }
            }
            e.op = id;
            c->op_arity[id] = (uint8_t)f.inputs.size();
            c->op_tt[id] = f.tt;
        } else {
            return ok = err->set(DP_EPARSE, "unknown library statement", ln);
        }
        if (lib->count(name)) return ok = err->set(DP_EPARSE, "library cell defined twice: " + name, ln);
        (*lib)[name] = std::move(e);
        return true;
    });
    return ok;
}

}  // namespace

extern "C" dp_status dp_compile(const char *netlist, size_t netlist_len, const char *library, size_t library_len,
                                dp_compiled **out, char *errbuf, size_t errlen) {
    Err err;
    auto fail = [&](dp_status code) {
        if (errbuf && errlen) std::snprintf(errbuf, errlen, "%s", err.msg.c_str());
        return code;
    };
    if (!out || (!netlist && netlist_len) || (!library && library_len)) {
        err.set(DP_EINVAL, "NULL argument");
        return fail(DP_EINVAL);
    }
    *out = nullptr;
    dp_compiled *c = new (std::nothrow) dp_compiled();
    if (!c) { err.set(DP_ENOMEM, "out of memory"); return fail(DP_ENOMEM); }
    try {
        for (int i = 0; i < 256; i++) { c->bc_offset[i] = -1; c->bc_length[i] = 0; }
        std::unordered_map<std::string, LibEntry> lib;
        if (!parse_library(std::string_view(library, library_len), &lib, c, &err)) {
            delete c;
            return fail(err.code);
        }
        std::unordered_map<std::string_view, const LibEntry *> libv;
        for (auto &kv : lib) libv[kv.first] = &kv.second;

        std::string_view text(netlist, netlist_len);
        // ---- pass 1: count
        int64_t nnet = 0, ncell = 0;
        for_lines(text, [&](std::string_view line, long) {
            size_t i = 0;
            while (i < line.size() && (line[i] == ' ' || line[i] == '\t')) i++;
            std::string_view l = line.substr(i);
            if (l.substr(0, 4) == "net ") nnet++;
            else if (l.substr(0, 5) == "cell ") ncell++;
            return true;
        });
        if (nnet > dp::kMaxNets) {
            err.set(DP_EUNSUPPORTED, "more than 2^24-1 nets");
            delete c;
            return fail(DP_EUNSUPPORTED);
        }
        std::unordered_map<std::string_view, int32_t> nets;
        nets.reserve((size_t)nnet * 2 + 16);
        std::vector<float> wire;
        wire.reserve((size_t)nnet);
        std::vector<float> dffcap;
        std::vector<int32_t> driver;   // -1 none, -2 startpoint, else user cell
        std::vector<int32_t> start_net;
        std::vector<const LibEntry *> cell_lib;
        std::vector<int32_t> cell_in;  // 4 per user cell (user net ids), -1 unused
        std::vector<int32_t> cell_out;
        cell_lib.reserve((size_t)ncell);
        cell_in.reserve((size_t)ncell * 4);
        cell_out.reserve((size_t)ncell);
        bool ok = true;
        for_lines(text, [&](std::string_view line, long ln) {
            std::string_view tok[4 + 2 * dp::kMaxArity + 2];
            int n = split(line, tok, 4 + 2 * dp::kMaxArity + 2, nullptr);
            if (n == 0 || tok[0] == "design") return true;
            auto net_id = [&](std::string_view name) -> int32_t {
                auto it = nets.find(name);
                return it == nets.end() ? -1 : it->second;
            };
            if (tok[0] == "net") {
                float w;
                if (n != 3 || !parse_float(tok[2], &w)) return ok = err.set(DP_EPARSE, "bad net line", ln);
                if (!nets.emplace(tok[1], (int32_t)wire.size()).second)
                    return ok = err.set(DP_EPARSE, "net declared twice", ln);
                wire.push_back(w);
                dffcap.push_back(0.f);
                driver.push_back(-1);
            } else if (tok[0] == "input") {
                int32_t id = n == 2 ? net_id(tok[1]) : -1;
                if (id < 0) return ok = err.set(DP_EPARSE, "bad input line", ln);
                if (driver[id] != -1) return ok = err.set(DP_EPARSE, "net has two drivers", ln);
                driver[id] = -2;
                start_net.push_back(id);
            } else if (tok[0] == "output") {
                if (n != 2 || net_id(tok[1]) < 0) return ok = err.set(DP_EPARSE, "bad output line", ln);
            } else if (tok[0] == "dff") {
                auto it = n == 5 ? libv.find(tok[2]) : libv.end();
                if (it == libv.end() || !it->second->seq) return ok = err.set(DP_EPARSE, "bad dff line", ln);
                const LibEntry *L = it->second;
                int32_t d = -1, q = -1;
                for (int t = 3; t < 5; t++) {
                    size_t eq = tok[t].find('=');
                    if (eq == std::string_view::npos) return ok = err.set(DP_EPARSE, "bad dff pin", ln);
                    std::string_view pin = tok[t].substr(0, eq);
                    int32_t id = net_id(tok[t].substr(eq + 1));
                    if (pin == L->dpin) d = id;
                    else if (pin == L->out) q = id;
                }
                if (d < 0 || q < 0) return ok = err.set(DP_EPARSE, "bad dff pins", ln);
                if (driver[q] != -1) return ok = err.set(DP_EPARSE, "net has two drivers", ln);
                dffcap[d] += L->pincap;
                driver[q] = -2;
                start_net.push_back(q);
            } else if (tok[0] == "cell") {
                auto it = n >= 3 ? libv.find(tok[2]) : libv.end();
                if (it == libv.end() || it->second->seq) return ok = err.set(DP_EPARSE, "unknown cell type", ln);
                const LibEntry *L = it->second;
                int k = (int)L->pins.size();
                if (n != 3 + k + 1) return ok = err.set(DP_EPARSE, "wrong pin count", ln);
                int32_t slot[dp::kMaxArity] = {-1, -1, -1, -1};
                int32_t o = -1;
                for (int t = 3; t < n; t++) {
                    size_t eq = tok[t].find('=');
                    if (eq == std::string_view::npos) return ok = err.set(DP_EPARSE, "bad pin", ln);
                    std::string_view pin = tok[t].substr(0, eq);
                    int32_t id = net_id(tok[t].substr(eq + 1));
                    if (id < 0) return ok = err.set(DP_EPARSE, "unknown net", ln);
                    if (pin == L->out) {
                        if (o >= 0) return ok = err.set(DP_EPARSE, "output pin twice", ln);
                        o = id;
                        continue;
                    }
                    int j = -1;
                    for (int q = 0; q < k; q++) if (L->pins[q] == pin) j = q;
                    if (j < 0 || slot[j] >= 0) return ok = err.set(DP_EPARSE, "bad or repeated input pin", ln);
                    slot[j] = id;
                }
                if (o < 0) return ok = err.set(DP_EPARSE, "output pin missing", ln);
                if (driver[o] != -1) return ok = err.set(DP_EPARSE, "net has two drivers", ln);
                driver[o] = (int32_t)cell_lib.size();
                cell_lib.push_back(L);
                for (int j = 0; j < dp::kMaxArity; j++) cell_in.push_back(slot[j]);
                cell_out.push_back(o);
            } else {
                return ok = err.set(DP_EPARSE, "unknown statement", ln);
            }
            return true;
        });
        if (!ok) { delete c; return fail(err.code); }
        const int64_t nn = (int64_t)wire.size(), nc = (int64_t)cell_lib.size(), ns = (int64_t)start_net.size();
        for (int64_t u = 0; u < nn; u++)
            if (driver[u] == -1) {
                err.set(DP_EPARSE, "undriven net");
                delete c;
                return fail(DP_EPARSE);
            }
        // ---- levelize (Sec. III-A): level = 1 + max fanin level, startpoints 0
        std::vector<int32_t> sink_ptr(nn + 1, 0), sink_cell;
        std::vector<int32_t> indeg(nc, 0), level(nc, 0), netlev(nn, 0);
        int64_t nedge = 0;
        for (int64_t cu = 0; cu < nc; cu++)
            for (int j = 0; j < dp::kMaxArity; j++) {
                int32_t u = cell_in[cu * 4 + j];
                if (u < 0) continue;
                nedge++;
                sink_ptr[u + 1]++;
                if (driver[u] >= 0) indeg[cu]++;
            }
        for (int64_t u = 0; u < nn; u++) sink_ptr[u + 1] += sink_ptr[u];
        sink_cell.resize((size_t)nedge);
        {
            std::vector<int32_t> fill(sink_ptr.begin(), sink_ptr.end() - 1);
            for (int64_t cu = 0; cu < nc; cu++)
                for (int j = 0; j < dp::kMaxArity; j++) {
                    int32_t u = cell_in[cu * 4 + j];
                    if (u >= 0) sink_cell[fill[u]++] = (int32_t)cu;
                }
        }
        std::vector<int32_t> queue;
        queue.reserve((size_t)nc);
        for (int64_t cu = 0; cu < nc; cu++) if (indeg[cu] == 0) queue.push_back((int32_t)cu);
        int32_t depth = 0;
        for (size_t h = 0; h < queue.size(); h++) {
            int32_t cu = queue[h];
            int32_t l = 0;
            for (int j = 0; j < dp::kMaxArity; j++) {
                int32_t u = cell_in[(size_t)cu * 4 + j];
                if (u >= 0 && netlev[u] > l) l = netlev[u];
            }
            level[cu] = l + 1;
            depth = std::max(depth, l + 1);
            int32_t o = cell_out[cu];
            netlev[o] = l + 1;
            for (int32_t s = sink_ptr[o]; s < sink_ptr[o + 1]; s++)
                if (--indeg[sink_cell[s]] == 0) queue.push_back(sink_cell[s]);
        }
        if ((int64_t)queue.size() != nc) {
            err.set(DP_ECYCLE, "combinational cycle");
            delete c;
            return fail(DP_ECYCLE);
        }
        // ---- renumber: level-major, logic id inside a level, then cell order
        std::vector<int32_t> order((size_t)nc);
        {
            std::vector<int64_t> cnt((size_t)256 * (depth + 1) + 1, 0);
            auto key = [&](int64_t cu) { return (int64_t)level[cu] * 256 + cell_lib[cu]->op; };
            for (int64_t cu = 0; cu < nc; cu++) cnt[key(cu) + 1]++;
            for (size_t i = 1; i < cnt.size(); i++) cnt[i] += cnt[i - 1];
            for (int64_t cu = 0; cu < nc; cu++) order[cnt[key(cu)]++] = (int32_t)cu;
        }
        c->n_nets = nn; c->n_start = ns; c->n_cells = nc; c->n_edges = nedge; c->n_levels = depth;
        c->lvl_ptr.assign((size_t)depth + 1, 0);
        c->cell_of_user.assign((size_t)nc, 0);
        c->user_of_cell.assign((size_t)nc, 0);
        for (int64_t ic = 0; ic < nc; ic++) {
            int32_t cu = order[ic];
            c->cell_of_user[cu] = (int32_t)ic;
            c->user_of_cell[ic] = cu;
            c->lvl_ptr[level[cu]] = (int32_t)(ic + 1);
        }
        for (int l = 1; l <= depth; l++) c->lvl_ptr[l] = std::max(c->lvl_ptr[l], c->lvl_ptr[l - 1]);
        c->net_of_user.assign((size_t)nn, 0);
        c->user_of_net.assign((size_t)nn, 0);
        for (int64_t k = 0; k < ns; k++) c->net_of_user[start_net[k]] = (int32_t)k;
        for (int64_t cu = 0; cu < nc; cu++) c->net_of_user[cell_out[cu]] = (int32_t)(ns + c->cell_of_user[cu]);
        for (int64_t u = 0; u < nn; u++) c->user_of_net[c->net_of_user[u]] = (int32_t)u;
        // ---- fanin records, caps
        c->fanin.assign((size_t)nc * 4, dp::kNetMask);
        c->pincap.assign((size_t)nc, 0.f);
        bool used[256] = {false};
        for (int64_t ic = 0; ic < nc; ic++) {
            int32_t cu = order[ic];
            const LibEntry *L = cell_lib[cu];
            used[L->op] = true;
            for (int j = 0; j < dp::kMaxArity; j++) {
                int32_t u = cell_in[(size_t)cu * 4 + j];
                if (u >= 0) c->fanin[ic * 4 + j] = (uint32_t)c->net_of_user[u];
            }
            c->fanin[ic * 4] = (c->fanin[ic * 4] & dp::kNetMask) | ((uint32_t)L->op << 24);
            c->pincap[ic] = L->pincap;
        }
        c->n_ops = 0;
        for (int i = 0; i < 256; i++) c->n_ops += used[i];
        c->base_cap.assign((size_t)nn, 0.f);
        for (int64_t u = 0; u < nn; u++) c->base_cap[c->net_of_user[u]] = wire[u] + dffcap[u];
        // ---- transposed fanout CSR, edges ascending within each net
        c->fout_ptr.assign((size_t)nn + 1, 0);
        for (int64_t ic = 0; ic < nc; ic++)
            for (int j = 0; j < dp::kMaxArity; j++) {
                uint32_t n = c->fanin[ic * 4 + j] & dp::kNetMask;
                if (j < c->op_arity[c->fanin[ic * 4] >> 24]) c->fout_ptr[n + 1]++;
            }
        for (int64_t n = 0; n < nn; n++) c->fout_ptr[n + 1] += c->fout_ptr[n];
        c->fout_edge.assign((size_t)nedge, 0);
        c->edge_fpos.assign((size_t)nc * 4, -1);
        {
            std::vector<int32_t> fill(c->fout_ptr.begin(), c->fout_ptr.end() - 1);
            for (int64_t ic = 0; ic < nc; ic++)
                for (int j = 0; j < dp::kMaxArity; j++) {
                    uint32_t n = c->fanin[ic * 4 + j] & dp::kNetMask;
                    if (j < c->op_arity[c->fanin[ic * 4] >> 24]) {
                        c->edge_fpos[ic * 4 + j] = fill[n];
                        c->fout_edge[fill[n]++] = (int32_t)(ic * 4 + j);
                    }
                }
        }
    } catch (const std::bad_alloc &) {
        delete c;
        err.set(DP_ENOMEM, "out of memory");
        return fail(DP_ENOMEM);
    }
    *out = c;
    return DP_OK;
}

extern "C" void dp_compiled_free(dp_compiled *c) { delete c; }

extern "C" dp_status dp_compiled_info(const dp_compiled *c, dp_info *info) {
    if (!c || !info) return DP_EINVAL;
    info->n_nets = c->n_nets;
    info->n_start = c->n_start;
    info->n_cells = c->n_cells;
    info->n_edges = c->n_edges;
    info->n_levels = c->n_levels;
    info->n_ops = c->n_ops;
    info->device_bytes = 0;
    info->block_threads = 0;
    info->cluster_threads = 0;
    return DP_OK;
}

extern "C" dp_status dp_compiled_view_get(const dp_compiled *c, dp_compiled_view *v) {
    if (!c || !v) return DP_EINVAL;
    v->lvl_ptr = c->lvl_ptr.data();
    v->fanin = c->fanin.data();
    v->fout_ptr = c->fout_ptr.data();
    v->fout_edge = c->fout_edge.data();
    v->net_of_user = c->net_of_user.data();
    v->cell_of_user = c->cell_of_user.data();
    v->base_cap = c->base_cap.data();
    v->pincap = c->pincap.data();
    v->op_arity = c->op_arity;
    v->op_tt = c->op_tt;
    v->bc_ops = c->bc_ops.data();
    v->bc_args = c->bc_args.data();
    v->bc_offset = c->bc_offset;
    v->bc_length = c->bc_length;
    v->n_bc = (int64_t)c->bc_ops.size();
    return DP_OK;
}

extern "C" dp_status dp_compile_function(const char *func, uint8_t *ops, int8_t *args, int32_t cap, int32_t *len,
                                         int32_t *n_inputs, uint16_t *tt, int32_t *logic_id) {
    if (!func) return DP_EINVAL;
    dp::Function f;
    std::string err;
    if (!dp::compile_function(func, &f, &err)) return DP_EPARSE;
    for (int32_t i = 0; i < (int32_t)f.ops.size() && i < cap; i++) {
        if (ops) ops[i] = f.ops[i];
        if (args) args[i] = f.args[i];
    }
    if (len) *len = (int32_t)f.ops.size();
    if (n_inputs) *n_inputs = (int32_t)f.inputs.size();
    if (tt) *tt = f.tt;
    if (logic_id) *logic_id = f.logic_id;
    return DP_OK;
}
