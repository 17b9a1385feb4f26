// Host side of the C ABI: kernel text parsing (loop domain, instruction,
// assumptions; Section 2.1), kernel printing, descriptor validation and
// dispatch to the CUDA kernels.  No device memory is allocated here.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <array>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "lc_internal.h"



namespace lc {

// ------------------------------------------------------------------ errors

static thread_local int g_last_cuda_error = 0;

lc_status cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int)e;
    return LC_ERR_CUDA;
}

// Device error word: set by bounded waits that give up.  Its device address is
// looked up once per device and passed to kernels as a parameter.
__device__ unsigned int g_device_error_word;

static std::mutex g_dev_mu;
static std::map<int, unsigned int *> g_err_ptr;
static std::map<int, int> g_sm_count;
static std::map<int, size_t> g_smem_optin;

unsigned int *error_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return nullptr;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_err_ptr.find(dev);
    if (it != g_err_ptr.end())
        return it->second;
    unsigned int *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, g_device_error_word) != cudaSuccess)
        return nullptr;
    g_err_ptr[dev] = p;
    return p;
}

int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_sm_count.find(dev);
    if (it != g_sm_count.end())
        return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    g_sm_count[dev] = n;
    return n;
}

size_t smem_optin_limit()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_smem_optin.find(dev);
    if (it != g_smem_optin.end())
        return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    g_smem_optin[dev] = (size_t)n;
    return (size_t)n;
}

int current_cc(int *major, int *minor)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return -1;
    if (cudaDeviceGetAttribute(major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
        return -1;
    if (cudaDeviceGetAttribute(minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return -1;
    return 0;
}

// ------------------------------------------------------------------ tokenizer

struct Tok {
    enum Kind { ID, INT, NUM, OP, END } kind;
    std::string s;
    long long v = 0;
    double d = 0.0;  // NUM: a literal with a fraction or an exponent
};

static bool tokenize(const char *text, std::vector<Tok> &out)
{
    out.clear();
    const char *p = text;
    while (*p) {
        unsigned char c = (unsigned char)*p;
        if (isspace(c)) {
            ++p;
            continue;
        }
        if (isalpha(c) || c == '_') {
            const char *b = p;
            while (isalnum((unsigned char)*p) || *p == '_')
                ++p;
            out.push_back({Tok::ID, std::string(b, p)});
            continue;
        }
        if (isdigit(c) || (c == '.' && isdigit((unsigned char)p[1]))) {
            // an integer, or a decimal literal with a fraction and/or an exponent
            const char *b = p;
            bool real = false;
            while (isdigit((unsigned char)*p))
                ++p;
            if (*p == '.') {
                real = true;
                ++p;
                while (isdigit((unsigned char)*p))
                    ++p;
            }
            if ((*p == 'e' || *p == 'E') &&
                (isdigit((unsigned char)p[1]) || ((p[1] == '-' || p[1] == '+') && isdigit((unsigned char)p[2])))) {
                real = true;
                p += 2;
                while (isdigit((unsigned char)*p))
                    ++p;
            }
            const std::string lit(b, p);
            if (real) {
                Tok t{Tok::NUM, lit};
                t.d = strtod(lit.c_str(), nullptr);
                out.push_back(t);
            } else {
                if (lit.size() > 15)
                    return false;
                Tok t{Tok::INT, lit};
                t.v = strtoll(lit.c_str(), nullptr, 10);
                out.push_back(t);
            }
            continue;
        }
        if ((p[0] == '<' || p[0] == '>' || p[0] == '=') && p[1] == '=') {
            out.push_back({Tok::OP, std::string(p, p + 2)});
            p += 2;
            continue;
        }
        if (strchr("{}[]():,<>=*-+/", c)) {
            out.push_back({Tok::OP, std::string(1, (char)c)});
            ++p;
            continue;
        }
        return false;
    }
    out.push_back({Tok::END, ""});
    return true;
}

struct Cursor {
    const std::vector<Tok> &t;
    size_t i = 0;
    explicit Cursor(const std::vector<Tok> &tt) : t(tt) {}
    const Tok &peek(size_t k = 0) const { return t[std::min(i + k, t.size() - 1)]; }
    bool op(const char *s)
    {
        if (peek().kind == Tok::OP && peek().s == s) {
            ++i;
            return true;
        }
        return false;
    }
    bool id(std::string &s)
    {
        if (peek().kind == Tok::ID) {
            s = peek().s;
            ++i;
            return true;
        }
        return false;
    }
    bool integer(long long &v)
    {
        bool neg = false;
        size_t save = i;
        if (op("-"))
            neg = true;
        if (peek().kind == Tok::INT) {
            v = neg ? -peek().v : peek().v;
            ++i;
            return true;
        }
        i = save;
        return false;
    }
    bool end() const { return peek().kind == Tok::END; }
};

// One side of a comparison chain: an integer, "P" or "P - 1", or a list of inames.
struct Operand {
    enum Kind { INT, PARAM, NAMES } kind;
    long long v = 0;
    std::string param;
    long long param_offset = 0;  // P + offset
    std::vector<std::string> names;
};

static bool parse_operand(Cursor &c, Operand &o)
{
    long long v;
    if (c.integer(v)) {
        o.kind = Operand::INT;
        o.v = v;
        return true;
    }
    std::string s;
    if (!c.id(s))
        return false;
    o.names = {s};
    if (c.op("-") || (c.peek().kind == Tok::OP && c.peek().s == "+")) {
        bool minus = c.t[c.i - 1].s == "-";
        if (!minus)
            c.op("+");
        long long k;
        if (c.peek().kind != Tok::INT)
            return false;
        k = c.peek().v;
        ++c.i;
        o.kind = Operand::PARAM;
        o.param = s;
        o.param_offset = minus ? -k : k;
        return true;
    }
    while (c.op(",")) {
        if (!c.id(s))
            return false;
        o.names.push_back(s);
    }
    o.kind = Operand::NAMES;
    return true;
}

static bool is_cmp(const Cursor &c)
{
    const Tok &t = c.peek();
    return t.kind == Tok::OP && (t.s == "<" || t.s == "<=" || t.s == ">" || t.s == ">=");
}

// Parse "{ [a,b,...] : chain and chain ... }" with an optional "[P,...] ->" prefix.
static bool parse_domain(const char *text, Kernel &K, std::string &why)
{
    std::vector<Tok> toks;
    if (!tokenize(text, toks)) {
        why = "domain: bad character";
        return false;
    }
    Cursor c(toks);
    if (c.peek().kind == Tok::OP && c.peek().s == "[") {
        // parameter list "[F, E, N] ->"
        c.op("[");
        std::string s;
        while (c.id(s))
            if (!c.op(","))
                break;
        if (!c.op("]") || !c.op("-") || !c.op(">")) {
            why = "domain: bad parameter list";
            return false;
        }
    }
    if (!c.op("{") || !c.op("[")) {
        why = "domain: expected '{ ['";
        return false;
    }
    std::string s;
    while (c.id(s)) {
        K.inames.push_back(s);
        if (!c.op(","))
            break;
    }
    if (!c.op("]") || !c.op(":")) {
        why = "domain: expected '] :'";
        return false;
    }
    std::map<std::string, int> lower;          // iname -> 1 if lower bound 0 seen
    std::map<std::string, std::string> upper;  // iname -> bounding parameter
    for (;;) {
        std::vector<Operand> ops;
        std::vector<std::string> cmps;
        Operand o;
        if (!parse_operand(c, o)) {
            why = "domain: expected a constraint";
            return false;
        }
        ops.push_back(o);
        while (is_cmp(c)) {
            cmps.push_back(c.peek().s);
            ++c.i;
            Operand o2;
            if (!parse_operand(c, o2)) {
                why = "domain: bad constraint operand";
                return false;
            }
            ops.push_back(o2);
        }
        if (cmps.empty()) {
            why = "domain: constraint without comparison";
            return false;
        }
        for (size_t k = 0; k < cmps.size(); ++k) {
            Operand L = ops[k], R = ops[k + 1];
            std::string op = cmps[k];
            // normalise to L (< | <=) R
            if (op == ">" || op == ">=") {
                std::swap(L, R);
                op = op == ">" ? "<" : "<=";
            }
            auto param_of = [&](const Operand &x, long long &off, std::string &p) {
                if (x.kind == Operand::PARAM) {
                    p = x.param;
                    off = x.param_offset;
                    return true;
                }
                if (x.kind == Operand::NAMES && x.names.size() == 1 &&
                    std::find(K.inames.begin(), K.inames.end(), x.names[0]) == K.inames.end()) {
                    p = x.names[0];
                    off = 0;
                    return true;
                }
                return false;
            };
            if (L.kind == Operand::INT && R.kind == Operand::NAMES) {
                // lower bound: 0 <= x  or  -1 < x
                bool ok = (op == "<=" && L.v == 0) || (op == "<" && L.v == -1);
                if (!ok) {
                    why = "domain: every lower bound must be 0";
                    return false;
                }
                for (auto &n : R.names)
                    lower[n] = 1;
                continue;
            }
            std::string p;
            long long off = 0;
            if (L.kind == Operand::NAMES && param_of(R, off, p) &&
                std::find(K.inames.begin(), K.inames.end(), L.names[0]) != K.inames.end()) {
                bool ok = (op == "<" && off == 0) || (op == "<=" && off == -1);
                if (!ok) {
                    why = "domain: upper bounds must read x < P or x <= P - 1";
                    return false;
                }
                for (auto &n : L.names) {
                    if (upper.count(n)) {
                        why = "domain: iname bounded twice";
                        return false;
                    }
                    upper[n] = p;
                }
                continue;
            }
            why = "domain: unsupported constraint";
            return false;
        }
        std::string kw;
        if (c.peek().kind == Tok::ID && c.peek().s == "and") {
            ++c.i;
            continue;
        }
        break;
    }
    if (!c.op("}") || !c.end()) {
        why = "domain: expected '}'";
        return false;
    }
    std::set<std::string> uniq(K.inames.begin(), K.inames.end());
    if (uniq.size() != K.inames.size()) {
        why = "domain: repeated iname";
        return false;
    }
    for (auto &n : K.inames) {
        if (!lower.count(n) || !upper.count(n)) {
            why = "domain: iname " + n + " lacks a bound";
            return false;
        }
        if (uniq.count(upper[n])) {
            why = "domain: bound must be a parameter";
            return false;
        }
        K.bounds.push_back(upper[n]);
    }
    for (auto &kv : lower)
        if (!uniq.count(kv.first)) {
            why = "domain: bound on unknown iname";
            return false;
        }
    return true;
}

struct Access {
    std::string name;
    std::vector<std::string> idx;
};

static bool parse_access(Cursor &c, Access &a)
{
    if (!c.id(a.name) || !c.op("["))
        return false;
    std::string s;
    while (c.id(s)) {
        a.idx.push_back(s);
        if (!c.op(","))
            break;
    }
    return c.op("]");
}

// Parse "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])" (or the F = 1 form) and assign roles.
static bool parse_instruction(const char *text, Kernel &K, std::string &why)
{
    std::vector<Tok> toks;
    if (!tokenize(text, toks)) {
        why = "instruction: bad character";
        return false;
    }
    Cursor c(toks);
    Access lhs, x, y;
    std::string red, sum;
    if (!parse_access(c, lhs) || !c.op("=")) {
        why = "instruction: expected 'out[...] ='";
        return false;
    }
    if (!c.id(sum) || sum != "sum" || !c.op("(") || !c.id(red) || !c.op(",")) {
        why = "instruction: expected 'sum(j, ...)'";
        return false;
    }
    if (!parse_access(c, x) || !c.op("*") || !parse_access(c, y) || !c.op(")") || !c.end()) {
        why = "instruction: expected a product of two array accesses";
        return false;
    }
    const bool multi = lhs.idx.size() == 3;
    if (!(lhs.idx.size() == 3 || lhs.idx.size() == 2)) {
        why = "instruction: output must have 2 or 3 indices";
        return false;
    }
    const size_t dn = multi ? 3 : 2;
    Access *Dp = nullptr, *Up = nullptr;
    if (x.idx.size() == dn && y.idx.size() == 2 && dn == 3) {
        Dp = &x;
        Up = &y;
    } else if (y.idx.size() == dn && x.idx.size() == 2 && dn == 3) {
        Dp = &y;
        Up = &x;
    } else if (dn == 2 && x.idx.size() == 2 && y.idx.size() == 2) {
        // D[i,j] * u[e,j]: D's first index is the output's last.
        const std::string &i = lhs.idx[1];
        if (x.idx[0] == i) {
            Dp = &x;
            Up = &y;
        } else {
            Dp = &y;
            Up = &x;
        }
    } else {
        why = "instruction: operand ranks do not match a contraction";
        return false;
    }
    std::string f = multi ? lhs.idx[0] : "", e = lhs.idx[multi ? 1 : 0], i = lhs.idx[multi ? 2 : 1];
    std::vector<std::string> dwant = multi ? std::vector<std::string>{f, i, red}
                                           : std::vector<std::string>{i, red};
    if (Dp->idx != dwant || Up->idx != std::vector<std::string>{e, red}) {
        why = "instruction: index structure is not out[f,e,i] = sum(j, D[f,i,j]*u[e,j])";
        return false;
    }
    std::vector<std::string> used = {e, i, red};
    if (multi)
        used.push_back(f);
    std::set<std::string> su(used.begin(), used.end());
    if (su.size() != used.size()) {
        why = "instruction: repeated iname";
        return false;
    }
    std::set<std::string> dom(K.inames.begin(), K.inames.end());
    if (su != dom) {
        why = "instruction: inames differ from the domain's";
        return false;
    }
    if (lhs.name == Dp->name || lhs.name == Up->name || Dp->name == Up->name) {
        why = "instruction: arrays must be distinct";
        return false;
    }
    auto bound = [&](const std::string &n) {
        size_t k = std::find(K.inames.begin(), K.inames.end(), n) - K.inames.begin();
        return K.bounds[k];
    };
    if (bound(i) != bound(red)) {
        why = "instruction: i and j must share one bound (square operators)";
        return false;
    }
    std::set<std::string> params = {bound(e), bound(i)};
    if (multi)
        params.insert(bound(f));
    if (params.size() != (multi ? 3u : 2u)) {
        why = "instruction: F, E and N must be distinct parameters";
        return false;
    }
    K.out_name = lhs.name;
    K.d_name = Dp->name;
    K.u_name = Up->name;
    K.f_iname = f;
    K.e_iname = e;
    K.i_iname = i;
    K.j_iname = red;
    K.F_param = multi ? bound(f) : "";
    K.E_param = bound(e);
    K.N_param = bound(i);
    return true;
}

// Parse the volume derivative with per-element geometric factors,
//   "out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*u[e,j])"
// (the three factors in any order): the reference derivatives sum_j D[f,i,j] u[e,j] mapped
// to physical coordinate d by the element's factors G[e,d,:]; d and f share the bound F.
static bool parse_geo_instruction(const char *text, Kernel &K, std::string &why)
{
    std::vector<Tok> toks;
    if (!tokenize(text, toks)) {
        why = "instruction: bad character";
        return false;
    }
    Cursor c(toks);
    Access lhs, fac[3];
    std::string sum, r1, r2;
    if (!parse_access(c, lhs) || !c.op("=") || !c.id(sum) || sum != "sum" || !c.op("(") || !c.op("(") ||
        !c.id(r1) || !c.op(",") || !c.id(r2) || !c.op(")") || !c.op(",")) {
        why = "instruction: expected 'out[d,e,i] = sum((f,j), ...)'";
        return false;
    }
    if (!parse_access(c, fac[0]) || !c.op("*") || !parse_access(c, fac[1]) || !c.op("*") ||
        !parse_access(c, fac[2]) || !c.op(")") || !c.end()) {
        why = "instruction: expected a product of three array accesses";
        return false;
    }
    if (lhs.idx.size() != 3) {
        why = "instruction: output must be out[d,e,i]";
        return false;
    }
    const std::string d = lhs.idx[0], e = lhs.idx[1], i = lhs.idx[2];
    Access *G = nullptr, *D = nullptr, *U = nullptr;
    for (Access &x : fac) {
        if (x.idx.size() == 2)
            U = &x;
        else if (x.idx.size() == 3 && x.idx[0] == e)
            G = &x;
        else if (x.idx.size() == 3)
            D = &x;
    }
    if (!G || !D || !U) {
        why = "instruction: factors must be G[e,d,f], D[f,i,j] and u[e,j]";
        return false;
    }
    std::string f = G->idx[2], j = U->idx[1];
    if (G->idx != std::vector<std::string>{e, d, f} || D->idx != std::vector<std::string>{f, i, j} ||
        U->idx != std::vector<std::string>{e, j} ||
        std::set<std::string>{r1, r2} != std::set<std::string>{f, j}) {
        why = "instruction: index structure is not out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*u[e,j])";
        return false;
    }
    std::set<std::string> su = {d, f, e, i, j};
    if (su.size() != 5 || su != std::set<std::string>(K.inames.begin(), K.inames.end())) {
        why = "instruction: inames differ from the domain's";
        return false;
    }
    std::set<std::string> names = {lhs.name, G->name, D->name, U->name};
    if (names.size() != 4) {
        why = "instruction: arrays must be distinct";
        return false;
    }
    auto bound = [&](const std::string &n) {
        return K.bounds[std::find(K.inames.begin(), K.inames.end(), n) - K.inames.begin()];
    };
    if (bound(d) != bound(f) || bound(i) != bound(j) ||
        std::set<std::string>{bound(f), bound(e), bound(i)}.size() != 3) {
        why = "instruction: d and f must share F, i and j must share N, and F, E, N must differ";
        return false;
    }
    K.kind = KIND_GEO;
    K.out_name = lhs.name;
    K.g_name = G->name;
    K.d_name = D->name;
    K.u_name = U->name;
    K.d_iname = d;
    K.f_iname = f;
    K.e_iname = e;
    K.i_iname = i;
    K.j_iname = j;
    K.F_param = bound(f);
    K.E_param = bound(e);
    K.N_param = bound(i);
    return true;
}

// Surface lift of the dG operator, in exactly this form (names free, bound on first use):
//   "out[e,i] = sum((f,p), L[i,f,p]*s[e,f]*(u[e,fmask[f,p]] - u[vmapP[e,f,p]]))"
// over { [e,i,f,p] : ... }: the jump between the interior trace u[e, fmask[f,p]] and the
// exterior trace u[vmapP[e,f,p]] (u read as a flat array through the map), scaled per face,
// lifted to the volume nodes.
static bool parse_lift_instruction(const char *text, Kernel &K, std::string &why)
{
    std::vector<Tok> toks;
    if (!tokenize(text, toks)) {
        why = "instruction: bad character";
        return false;
    }
    static const char *pat[] = {"$out", "[", "$e", ",", "$i", "]", "=", "#sum", "(", "(", "$f", ",", "$p", ")", ",",
                                "$L", "[", "$i", ",", "$f", ",", "$p", "]", "*", "$s", "[", "$e", ",", "$f", "]", "*",
                                "(", "$u", "[", "$e", ",", "$fm", "[", "$f", ",", "$p", "]", "]", "-", "$u", "[",
                                "$vm", "[", "$e", ",", "$f", ",", "$p", "]", "]", ")", ")"};
    std::map<std::string, std::string> bind;
    size_t t = 0;
    for (const char *q : pat) {
        if (t >= toks.size())
            return false;
        const Tok &tk = toks[t++];
        if (q[0] == '$') {
            if (tk.kind != Tok::ID)
                return false;
            auto it = bind.find(q);
            if (it == bind.end())
                bind[q] = tk.s;
            else if (it->second != tk.s)
                return false;
        } else if (q[0] == '#') {
            if (tk.kind != Tok::ID || tk.s != q + 1)
                return false;
        } else if (tk.kind != Tok::OP || tk.s != q) {
            return false;
        }
    }
    if (toks[t].kind != Tok::END)
        return false;
    const std::set<std::string> in = {bind["$e"], bind["$i"], bind["$f"], bind["$p"]};
    if (in.size() != 4 || in != std::set<std::string>(K.inames.begin(), K.inames.end())) {
        why = "instruction: inames differ from the domain's";
        return false;
    }
    const std::set<std::string> arrays = {bind["$out"], bind["$L"], bind["$s"], bind["$u"], bind["$fm"], bind["$vm"]};
    if (arrays.size() != 6) {
        why = "instruction: arrays must be distinct";
        return false;
    }
    auto bound = [&](const std::string &n) {
        return K.bounds[std::find(K.inames.begin(), K.inames.end(), n) - K.inames.begin()];
    };
    if (std::set<std::string>{bound(bind["$e"]), bound(bind["$i"]), bound(bind["$f"]), bound(bind["$p"])}.size() != 4) {
        why = "instruction: E, N, Nf and Nfp must be distinct parameters";
        return false;
    }
    K.kind = KIND_LIFT;
    K.out_name = bind["$out"];
    K.d_name = bind["$L"];
    K.s_name = bind["$s"];
    K.u_name = bind["$u"];
    K.fmask_name = bind["$fm"];
    K.vmap_name = bind["$vm"];
    K.e_iname = bind["$e"];
    K.i_iname = bind["$i"];
    K.f_iname = bind["$f"];
    K.p_iname = bind["$p"];
    K.E_param = bound(bind["$e"]);
    K.N_param = bound(bind["$i"]);
    K.Nf_param = bound(bind["$f"]);
    K.Nfp_param = bound(bind["$p"]);
    return true;
}

// Elementwise instruction "lhs[i0, i1] = expr" over a domain of one or two inames: expr is
// built from +, -, *, / (left-associative, * and / binding tighter), unary minus,
// parentheses, decimal literals, scalar parameters (unindexed names) and array accesses
// indexed by inames in domain order (a subset of them: broadcast along the others).
struct EwParser {
    Cursor &c;
    Kernel &K;
    std::string why;
    EwParser(Cursor &cc, Kernel &kk) : c(cc), K(kk) {}
    int add(EwNode n)
    {
        K.ew.nodes.push_back(n);
        return (int)K.ew.nodes.size() - 1;
    }
    int primary()
    {
        if (c.op("(")) {
            int e = expr();
            if (e < 0 || !c.op(")"))
                return -1;
            return e;
        }
        if (c.op("-")) {
            int a = primary();
            if (a < 0)
                return -1;
            EwNode n{EW_NEG};
            n.a = a;
            return add(n);
        }
        const Tok &t = c.peek();
        if (t.kind == Tok::INT || t.kind == Tok::NUM) {
            EwNode n{EW_CONST};
            n.val = t.kind == Tok::INT ? (double)t.v : t.d;
            ++c.i;
            return add(n);
        }
        std::string name;
        if (!c.id(name)) {
            why = "instruction: expected an operand";
            return -1;
        }
        if (std::find(K.inames.begin(), K.inames.end(), name) != K.inames.end()) {
            why = "instruction: inames are indices, not values";
            return -1;
        }
        if (!c.op("[")) {  // a scalar parameter
            auto it = std::find(K.ew.params.begin(), K.ew.params.end(), name);
            EwNode n{EW_PARAM};
            n.arg = (int)(it - K.ew.params.begin());
            if (it == K.ew.params.end())
                K.ew.params.push_back(name);
            return add(n);
        }
        std::vector<int> dims;
        std::string ix;
        while (c.id(ix)) {
            auto it = std::find(K.inames.begin(), K.inames.end(), ix);
            if (it == K.inames.end()) {
                why = "instruction: index is not an iname";
                return -1;
            }
            dims.push_back((int)(it - K.inames.begin()));
            if (!c.op(","))
                break;
        }
        if (!c.op("]") || dims.empty()) {
            why = "instruction: bad array access";
            return -1;
        }
        for (size_t q = 1; q < dims.size(); ++q)
            if (dims[q] <= dims[q - 1]) {
                why = "instruction: indices must follow the domain order";
                return -1;
            }
        int k = -1;
        for (size_t q = 0; q < K.ew.arrays.size(); ++q)
            if (K.ew.arrays[q].name == name)
                k = (int)q;
        if (k == 0) {
            why = "instruction: the output cannot be read";
            return -1;
        }
        if (k > 0 && K.ew.arrays[k].dims != dims) {
            why = "instruction: one array, two index lists";
            return -1;
        }
        if (k < 0) {
            K.ew.arrays.push_back({name, dims});
            k = (int)K.ew.arrays.size() - 1;
        }
        EwNode n{EW_LOAD};
        n.arg = k;
        return add(n);
    }
    int term()
    {
        int a = primary();
        while (a >= 0 && (c.peek().kind == Tok::OP && (c.peek().s == "*" || c.peek().s == "/"))) {
            const bool mul = c.peek().s == "*";
            ++c.i;
            int b = primary();
            if (b < 0)
                return -1;
            EwNode n{mul ? EW_MUL : EW_DIV};
            n.a = a;
            n.b = b;
            a = add(n);
        }
        return a;
    }
    int expr()
    {
        int a = term();
        while (a >= 0 && (c.peek().kind == Tok::OP && (c.peek().s == "+" || c.peek().s == "-"))) {
            const bool plus = c.peek().s == "+";
            ++c.i;
            int b = term();
            if (b < 0)
                return -1;
            EwNode n{plus ? EW_ADD : EW_SUB};
            n.a = a;
            n.b = b;
            a = add(n);
        }
        return a;
    }
};

static bool parse_elementwise(const char *text, Kernel &K, std::string &why)
{
    if (K.inames.empty() || K.inames.size() > 2) {
        why = "instruction: elementwise domains have one or two inames";
        return false;
    }
    std::vector<Tok> toks;
    if (!tokenize(text, toks)) {
        why = "instruction: bad character";
        return false;
    }
    Cursor c(toks);
    Access lhs;
    if (!parse_access(c, lhs) || !c.op("=") || lhs.idx != K.inames) {
        why = "instruction: the output must be indexed by every iname, in domain order";
        return false;
    }
    K.ew = Elementwise();
    std::vector<int> all;
    for (size_t d = 0; d < K.inames.size(); ++d)
        all.push_back((int)d);
    K.ew.arrays.push_back({lhs.name, all});
    EwParser P(c, K);
    K.ew.root = P.expr();
    if (K.ew.root < 0 || !c.end()) {
        why = P.why.empty() ? "instruction: trailing text" : P.why;
        return false;
    }
    if (K.ew.nodes.size() > 256 || K.ew.arrays.size() > 17 || K.ew.params.size() > 16) {
        why = "instruction: expression too large";
        return false;
    }
    std::set<std::string> bnd(K.bounds.begin(), K.bounds.end());
    if (bnd.size() != K.bounds.size()) {
        why = "instruction: each iname needs its own bound";
        return false;
    }
    for (const auto &p : K.ew.params) {
        if (bnd.count(p) || std::find(K.inames.begin(), K.inames.end(), p) != K.inames.end()) {
            why = "instruction: a parameter shadows a bound or an iname";
            return false;
        }
        for (const auto &a : K.ew.arrays)
            if (a.name == p) {
                why = "instruction: one name used as an array and as a scalar";
                return false;
            }
    }
    K.kind = KIND_ELEMENTWISE;
    K.out_name = lhs.name;
    return true;
}

static bool parse_assumptions(const char *text, Kernel &K, std::string &why)
{
    if (!text)
        return true;
    std::vector<Tok> toks;
    if (!tokenize(text, toks)) {
        why = "assumptions: bad character";
        return false;
    }
    Cursor c(toks);
    if (c.end())
        return true;
    std::set<std::string> params = {K.E_param, K.N_param};
    if (!K.F_param.empty())
        params.insert(K.F_param);
    if (K.kind == KIND_ELEMENTWISE || K.kind == KIND_LIFT)
        params = std::set<std::string>(K.bounds.begin(), K.bounds.end());
    for (;;) {
        Assumption a;
        if (!c.id(a.param) || !params.count(a.param)) {
            why = "assumptions: expected a parameter of the domain";
            return false;
        }
        if (c.peek().kind == Tok::ID && c.peek().s == "mod") {
            ++c.i;
            long long k, z;
            if (!c.integer(k) || k <= 0 || !c.op("=") || !c.integer(z) || z != 0) {
                why = "assumptions: expected 'P mod k = 0'";
                return false;
            }
            a.op = 0;
            a.k = k;
        } else {
            const std::string s = c.peek().s;
            if (c.peek().kind != Tok::OP) {
                why = "assumptions: expected a comparison";
                return false;
            }
            if (s == ">=") a.op = 1;
            else if (s == ">") a.op = 2;
            else if (s == "<=") a.op = 3;
            else if (s == "<") a.op = 4;
            else if (s == "=" || s == "==") a.op = 5;
            else {
                why = "assumptions: unknown comparison";
                return false;
            }
            ++c.i;
            if (!c.integer(a.k)) {
                why = "assumptions: expected an integer";
                return false;
            }
        }
        K.assumptions.push_back(a);
        if (c.peek().kind == Tok::ID && c.peek().s == "and") {
            ++c.i;
            continue;
        }
        break;
    }
    if (!c.end()) {
        why = "assumptions: trailing text";
        return false;
    }
    return true;
}

static bool assumptions_hold(const Kernel &K, long long E, long long N, long long F)
{
    for (const auto &a : K.assumptions) {
        long long v = a.param == K.E_param ? E : a.param == K.N_param ? N : F;
        bool ok = true;
        switch (a.op) {
        case 0: ok = (v % a.k) == 0; break;
        case 1: ok = v >= a.k; break;
        case 2: ok = v > a.k; break;
        case 3: ok = v <= a.k; break;
        case 4: ok = v < a.k; break;
        case 5: ok = v == a.k; break;
        }
        if (!ok)
            return false;
    }
    return true;
}

// True when the assumptions imply E mod m == 0.
static bool implies_E_multiple_of(const Kernel &K, long long m)
{
    for (const auto &a : K.assumptions)
        if (a.param == K.E_param && a.op == 0 && a.k % m == 0)
            return true;
    return false;
}

// ------------------------------------------------------------------ validation

// Warp shape WE x WC and column groups CG (a multiple of WC) covering C columns in one
// pass: the fewest padded columns within `max_threads` (and within `req_threads` when > 0:
// a CTA of that size whose surplus warps only help with loads) and the shared memory left
// for D^T after `fixed` bytes.
static bool simt_warp_shape(SimtGeom &g, int C, int N, int es, size_t fixed, size_t smem_cap, int max_threads,
                            int req_threads)
{
    const int ncg = (C + g.RC - 1) / g.RC;
    const int wcs[6] = {4, 2, 8, 1, 16, 32};
    long long best_waste = -1;
    for (int wc : wcs) {
        const int we = 32 / wc;
        if (g.EG % we != 0)
            continue;
        if (fixed + (size_t)N * g.RC * wc * es > smem_cap)
            continue;
        const long long cg_smem = (long long)((smem_cap - fixed) / ((size_t)N * g.RC * es));
        const int cap = req_threads > 0 ? std::min(max_threads, req_threads) : max_threads;
        long long cg = ((ncg + wc - 1) / wc) * (long long)wc;
        cg = std::min<long long>(cg, (cap / g.EG) / wc * (long long)wc);
        cg = std::min<long long>(cg, cg_smem / wc * (long long)wc);
        if (cg < wc)
            continue;
        const long long cw = cg * g.RC;
        if (cw < C)
            continue;  // the CTA's whole column block must fit one pass
        const long long waste = cw - C;
        if (best_waste < 0 || waste < best_waste) {
            best_waste = waste;
            g.WC = wc;
            g.CG = (int)cg;
        }
    }
    return best_waste >= 0;
}

// Apply the descriptor's grid bound (max_ctas > 0) to a grid of whole column-block sets:
// false if the bound is below one set or the grid does not fit an int.
static bool cap_grid(long long &grid, int nblocks, int max_ctas)
{
    if (max_ctas > 0) {
        if (max_ctas < nblocks)
            return false;
        grid = std::min<long long>(grid, (long long)max_ctas / nblocks * nblocks);
    }
    return grid <= 0x7fffffffLL;
}

struct Resolved {
    int engine, layout, precision;
    SimtGeom g;
    TcArgs tc;
    int tc_grid;
    KsArgs ks;     // K-split engine
    int ks_bm, ks_bk;
    int unroll, prefetch, tail_free;
    int warp_per;  // WARP engine: elements per warp step
};

static lc_status resolve(const Kernel &K, long long E, int N, int F, const lc_variant *v, Resolved &r,
                         bool need_device, int req_threads = 0)
{
    if (!v || v->struct_size != sizeof(lc_variant))
        return LC_ERR_INVALID_ARGUMENT;
    if (E < 0 || N < 1 || N > 256 || F < 1 || F > 8)
        return LC_ERR_INVALID_ARGUMENT;
    if (K.F_param.empty() && F != 1)
        return LC_ERR_INVALID_ARGUMENT;
    if (!assumptions_hold(K, E, N, F))
        return LC_ERR_ASSUMPTION;
    if (v->layout != LC_LAYOUT_ELEM_MAJOR && v->layout != LC_LAYOUT_NODE_MAJOR)
        return LC_ERR_INVALID_VARIANT;
    if (v->precision < LC_PREC_FP64 || v->precision > LC_PREC_BF16X3)
        return LC_ERR_INVALID_VARIANT;
    if (v->tail_free != 0 && v->tail_free != 1)
        return LC_ERR_INVALID_VARIANT;
    if (v->ctas_per_sm < 0 || v->ctas_per_sm > 32 || v->max_ctas < 0)
        return LC_ERR_INVALID_VARIANT;
    const bool geo = K.kind == KIND_GEO;
    if (geo) {
        // every operator in one column block (the epilogue mixes all F partial sums of a node);
        // kernel instances exist for F = 2 and 3; whole-tile staging slots
        if (v->engine != LC_ENGINE_TCGEN05 || F < 2 || F > 3 || !(v->split_i == 0 || v->split_i == F) ||
            !(v->store_rows == 0 || v->store_rows == 128))
            return LC_ERR_INVALID_VARIANT;
    }
    r.engine = v->engine;
    r.layout = v->layout;
    r.precision = v->precision;
    r.unroll = v->unroll;
    r.prefetch = v->prefetch_smem;
    r.tail_free = v->tail_free;
    if (v->tail_free && !implies_E_multiple_of(K, v->tile_e > 0 ? v->tile_e : 1))
        return LC_ERR_INVALID_VARIANT;  // the guard-free last tile needs "E mod tile_e = 0"
    const int sms = need_device ? sm_count() : 148;
    const size_t smem_cap = need_device ? smem_optin_limit() : 232448;
    if (need_device && (sms <= 0 || smem_cap == 0))
        return LC_ERR_NO_DEVICE;

    if (v->engine != LC_ENGINE_TCGEN05 &&
        (v->out_buffers != 0 || v->store_rows != 0 || v->mma_order != 0 || v->a_operand != 0))
        return LC_ERR_INVALID_VARIANT;
    if (v->engine == LC_ENGINE_SIMT) {
        if (v->precision != LC_PREC_FP32 && v->precision != LC_PREC_FP64)
            return LC_ERR_INVALID_VARIANT;
        const int VEC = v->precision == LC_PREC_FP64 ? 2 : 4;
        const int es = v->precision == LC_PREC_FP64 ? 8 : 4;
        SimtGeom &g = r.g;
        g.VEC = VEC;
        g.RE = v->elems_per_thread;
        g.RC = v->split_i;
        if (!(g.RE == VEC || g.RE == 2 * VEC) || !(g.RC == VEC || g.RC == 2 * VEC))
            return LC_ERR_INVALID_VARIANT;
        if (!(v->unroll == 1 || v->unroll == 2 || v->unroll == 4 || v->unroll == 8))
            return LC_ERR_INVALID_VARIANT;
        if (v->prefetch_smem != 0 && v->prefetch_smem != 1)
            return LC_ERR_INVALID_VARIANT;
        if (v->stages < 1 || v->stages > 2 || (!v->prefetch_smem && v->stages != 1))
            return LC_ERR_INVALID_VARIANT;
        if (v->tile_e <= 0 || v->tile_e % g.RE != 0)
            return LC_ERR_INVALID_VARIANT;
        g.TE = v->tile_e;
        g.EG = g.TE / g.RE;
        const int max_threads = g.RE * g.RC >= 64 ? 256 : 512;  // register budget per thread
        if (g.EG > max_threads)
            return LC_ERR_INVALID_VARIANT;
        g.stages = v->stages;
        const bool node = v->layout == LC_LAYOUT_NODE_MAJOR;
        // column blocks of G whole operators, one per CTA with its D^T resident: the most
        // operators per block that fit (fewer blocks re-reading the same u tile)
        bool fits = false;
        size_t fixed = 0;
        size_t fixed_u = 16;  // mbarriers + u tiles
        if (v->prefetch_smem)
            fixed_u += node ? (size_t)g.stages * N * g.TE * es
                            : (size_t)N * (g.TE + VEC) * es + (size_t)g.stages * g.TE * N * es;
        g.isplit = 0;
        for (int G = F; G >= 1 && !fits; --G) {
            fixed = fixed_u + (node ? 0 : (size_t)G * g.TE * N * es);  // + output staging
            if (simt_warp_shape(g, G * N, N, es, fixed, smem_cap, max_threads, req_threads)) {
                g.G = G;
                fits = true;
            }
        }
        // one operator's D^T does not fit: blocks of rows of one operator
        for (int parts = 2; parts <= N && !fits; ++parts) {
            const int w = (N + parts - 1) / parts;
            fixed = fixed_u + (node ? 0 : (size_t)g.TE * w * es);
            if (simt_warp_shape(g, w, N, es, fixed, smem_cap, max_threads, req_threads)) {
                g.G = 1;
                g.isplit = w;
                fits = true;
            }
        }
        if (!fits)
            return LC_ERR_INVALID_VARIANT;
        g.threads = g.EG * g.CG;
        g.CW = g.CG * g.RC;
        g.nchunks = g.isplit ? F * ((N + g.isplit - 1) / g.isplit) : (F + g.G - 1) / g.G;
        g.smem = fixed + (size_t)N * g.CW * es;
        if (g.smem > smem_cap || g.threads > max_threads || g.threads % 32 != 0)
            return LC_ERR_INVALID_VARIANT;
        g.bulk = v->prefetch_smem && (!node || E % VEC == 0);
        g.bulk_store = !node && ((E * (long long)N) % VEC == 0);
        g.ntiles = (E + g.TE - 1) / g.TE;
        long long grid = std::max<long long>(g.ntiles, 1) * g.nchunks;
        if (v->ctas_per_sm > 0)
            grid = std::min<long long>(grid, (long long)v->ctas_per_sm * sms);
        grid = std::max<long long>(grid / g.nchunks * g.nchunks, g.nchunks);  // whole column-block sets
        if (!cap_grid(grid, g.nchunks, v->max_ctas))
            return LC_ERR_INVALID_VARIANT;
        g.grid = (int)grid;
        return LC_OK;
    }
    if (v->engine == LC_ENGINE_TCGEN05) {
        if (v->precision != LC_PREC_BF16 && v->precision != LC_PREC_BF16X3)
            return LC_ERR_INVALID_VARIANT;
        // unroll = threads that share one tile row in the epilogue (1..4); the conversion
        // gets as many, up to 26 warps per CTA in all (unroll 4: two conversion threads);
        // elems_per_thread = K-block width (16, 32 or 64 bf16 = 32/64/128-byte swizzle rows),
        // K padded to a multiple of it; 1 = the widest block that divides K padded to 16
        const int kbw = v->elems_per_thread;
        if (v->tile_e != 128 || !(v->prefetch_smem == 1 || v->prefetch_smem == 2) ||
            !(kbw == 1 || kbw == 16 || kbw == 32 || kbw == 64) ||
            v->unroll < 1 || v->unroll > 4)
            return LC_ERR_INVALID_VARIANT;
        if (v->stages < 1 || v->stages > 3 || v->split_i < 0 || v->split_i > F || v->ctas_per_sm > 1 ||
            v->out_buffers < 0 || v->out_buffers > 4 ||
            !(v->store_rows == 0 || v->store_rows == 32 || v->store_rows == 64 || v->store_rows == 128))
            return LC_ERR_INVALID_VARIANT;
        const bool node = v->layout == LC_LAYOUT_NODE_MAJOR;
        const int NT = v->precision == LC_PREC_BF16X3 ? 3 : 1;
        if (v->mma_order < 0 || v->mma_order > 2 || (v->mma_order != 0 && NT != 3))
            return LC_ERR_INVALID_VARIANT;
        if (v->a_operand < 0 || v->a_operand > 2 || (v->a_operand == 2 && geo && NT != 1))
            return LC_ERR_INVALID_VARIANT;  // three-term A in tensor memory: not in the geometric-factor kernel
        TcArgs &t = r.tc;
        memset(&t, 0, sizeof t);
        t.N = N;
        t.F = F;
        t.E = E;
        t.Kt = (N + 15) / 16 * 16;
        if (kbw == 1) {
            t.Kp = t.Kt;
            t.KB = t.Kp % 64 == 0 ? 64 : (t.Kp % 32 == 0 ? 32 : 16);
        } else {
            t.KB = kbw;
            t.Kp = (t.Kt + kbw - 1) / kbw * kbw;
        }
        t.nkb = t.Kp / t.KB;
        if (t.nkb > 16)
            return LC_ERR_INVALID_VARIANT;  // more K-blocks than the kernel has barrier pairs for
        t.stages = v->stages;
        t.early_release = v->prefetch_smem == 2;
        t.threads_per_row = v->unroll;
        t.conv_threads_per_row = std::min(v->unroll, 6 - v->unroll);
        const size_t W = 2 * (size_t)t.KB;
        // rows per element-major bulk store: whole tiles of every operator of the block for
        // small N (few, large stores), else 32-row pieces of one operator at a time (the
        // stores stream, and the staging slots stay small)
        t.store_quarters = geo ? 4 : (v->store_rows ? v->store_rows / 32 : (N <= 48 ? 4 : 1));
        // a_tm: A terms in tensor memory (one accumulator region each: BF16, or BF16X3 with the
        // hi*hi products last), else in shared memory
        auto plan = [&](int G, TcArgs &q, bool a_tm) -> bool {
            q.G = G;
            // operator padding: 16 columns (16-column epilogue chunks), or 8 where that lets
            // the BF16X3 terms stack (2 CBp <= 256) or the block fit (CBp <= 256) at all
            auto cbp = [&](int np) { return (G * np + 15) / 16 * 16; };
            const int np16 = (N + 15) / 16 * 16, np8 = (N + 7) / 8 * 8;
            const bool want_stack = NT == 3 && v->mma_order != 2 && !a_tm;
            if (want_stack && 2 * cbp(np16) > 256 && 2 * cbp(np8) <= 256)
                q.Np = np8;
            else if ((NT == 3 || a_tm) && !want_stack && cbp(np8) < cbp(np16))
                q.Np = np8;  // one accumulator region: the narrowest padding (smaller B, fewer columns)
            else
                q.Np = cbp(np16) <= 256 ? np16 : np8;
            // three terms, whole-tile epilogue (node-major, or element-major stores of whole
            // tiles): the operators packed without padding where that narrows the MMAs, whose
            // time grows with their N (the epilogue chunks may then cross an operator's end)
            if (NT == 3 && !geo && (node || t.store_quarters == 4) && N >= 8 && cbp(N) < cbp(q.Np) &&
                (!want_stack || 2 * cbp(N) <= 256))
                q.Np = N;
            q.chunk = q.Np % 16 == 0 && !geo ? 16 : 8;
            q.CB = G * q.Np;
            q.CBp = cbp(q.Np);
            if (q.CBp > 256)
                return false;
            q.stack = want_stack && 2 * q.CBp <= 256;
            if (v->mma_order == 1 && !q.stack)
                return false;  // the stacked order needs 2 x MMA N <= 256
            q.tmem_cols = 32;
            while (q.tmem_cols < (q.stack ? 2 : 1) * q.CBp)
                q.tmem_cols *= 2;
            q.a_tmem = a_tm;
            q.a_cols = a_tm ? NT * q.Kt / 2 : 0;
            const int need = 2 * q.tmem_cols + q.abufs * q.a_cols;
            if (need > 512)
                return false;
            q.tmem_alloc = 32;
            while (q.tmem_alloc < need)
                q.tmem_alloc *= 2;
            size_t off = 0;
            off += (size_t)NT * q.nkb * q.CBp * W;                       // B terms
            off += a_tm ? 0 : (size_t)q.abufs * NT * q.nkb * 128 * W;  // A terms
            q.off_stage = (unsigned)off;
            off += (size_t)q.stages * 128 * N * 4;
            q.off_out = (unsigned)off;
            if (!node)  // staging slots: every operator of the block (4 quarters per store), else one
                off += (size_t)q.obufs * (q.store_quarters == 4 ? G : 1) * 128 * N * 4;
            off = (off + 15) / 16 * 16;
            q.off_bar = (unsigned)off;
            off += 1024;  // 10 mbarriers, TMEM address, abort flag; 2 x 2 x 16 A-block mbarriers
            // alignment slack; at least 120 KB so one CTA holds an SM (and its tensor memory)
            q.smem_bytes = (unsigned)std::max<size_t>(off + 1024, 120 * 1024);
            return q.smem_bytes <= smem_cap;
        };
        if (v->stages > 3)
            return LC_ERR_INVALID_VARIANT;
        // Shared-memory plan, in order of preference: the most operators per CTA (fewer
        // column blocks re-reading the same u tile), then at least two output staging
        // slots (the bulk stores of one slot overlap the staging of the next), then two A
        // buffers (conversion of tile k+1 overlaps the MMAs of tile k), then more slots.
        static const int combos[][2] = {{3, 2}, {2, 2}, {4, 1}, {3, 1}, {2, 1}, {1, 2}, {1, 1}};  // {slots, abufs}
        const int ncombos = (int)(sizeof combos / sizeof combos[0]);
        bool found = false;
        const int g_hi = v->split_i ? v->split_i : F, g_lo = geo ? F : (v->split_i ? v->split_i : 1);
        // the most operators per CTA first; for each, the planner's A placement first: tensor
        // memory for BF16 (it frees shared memory for stages and slots), shared memory for
        // BF16X3 (the stacked order needs both accumulators' columns, and a long chain of MMAs
        // reading A from tensor memory measured slower beside the epilogue's loads); BF16X3
        // takes tensor-memory A where no shared-memory plan fits (N above about 100)
        const bool tm_first = v->a_operand == 2 || (v->a_operand == 0 && NT == 1);
        for (int g = g_hi; g >= g_lo && !found; --g)
            for (int pass = 0; pass < 2 && !found; ++pass) {
                const bool a_tm = tm_first ? pass == 0 : pass == 1;
                if ((a_tm && v->a_operand == 1) || (!a_tm && v->a_operand == 2) || (a_tm && geo && NT != 1))
                    continue;
                for (int c = 0; c < ncombos && !found; ++c) {
                    TcArgs q = t;
                    q.obufs = node ? 1 : combos[c][0];
                    q.abufs = combos[c][1];
                    if (!node && v->out_buffers && q.obufs != v->out_buffers)
                        continue;
                    if (plan(g, q, a_tm)) {
                        t = q;
                        found = true;
                    }
                }
        }
        if (!found)
            return LC_ERR_INVALID_VARIANT;
        const int G = t.G;
        t.nblocks = (F + G - 1) / G;
        t.ntiles = (E + 127) / 128;
        // element-major whole-tile slots: the store warp issues the bulk stores and waits for
        // their reads, so the epilogue warps go on to the next tile at once
        t.store_warp = !node && t.store_quarters == 4;
        t.bulk_u = node ? (E % 4 == 0) : 1;
        t.bulk_store = !node && ((E * (long long)N) % 4 == 0);
        long long work = t.ntiles * t.nblocks;
        long long grid = std::min<long long>(work, (long long)sms);
        grid = std::max<long long>(grid / t.nblocks * t.nblocks, t.nblocks);
        if (!cap_grid(grid, t.nblocks, v->max_ctas))
            return LC_ERR_INVALID_VARIANT;
        r.tc_grid = (int)grid;
        return LC_OK;
    }
    if (v->engine == LC_ENGINE_KSPLIT) {
        // FP32; tile_e = BM (64 or 128), 8 x 8 register blocks, unroll = BK (the j chunk: 8
        // or 16), prefetch of u into shared memory with stages = 1 or 2 u buffers
        if (v->precision != LC_PREC_FP32 || v->tail_free || !(v->tile_e == 64 || v->tile_e == 128) ||
            v->elems_per_thread != 8 || v->split_i != 8 || !(v->unroll == 8 || v->unroll == 16) ||
            v->prefetch_smem != 1 || !(v->stages == 1 || v->stages == 2) || v->ctas_per_sm > 4)
            return LC_ERR_INVALID_VARIANT;
        KsArgs &k = r.ks;
        memset(&k, 0, sizeof k);
        const bool node = v->layout == LC_LAYOUT_NODE_MAJOR;
        const int BM = v->tile_e, BK = v->unroll;
        k.E = E;
        k.N = N;
        k.F = F;
        k.C = F * N;
        k.Kp = (N + BK - 1) / BK * BK;
        k.nkc = k.Kp / BK;
        k.nblocks = (k.C + 127) / 128;
        k.ntiles = (E + BM - 1) / BM;
        k.ubufs = v->stages;
        k.vec_u = node && E % 4 == 0;
        k.vec_out = node ? E % 4 == 0 : N % 4 == 0;
        r.ks_bm = BM;
        r.ks_bk = BK;
        const size_t smem = ks_smem_bytes(k.Kp, BM, BK, k.ubufs);
        if (smem > smem_cap)
            return LC_ERR_INVALID_VARIANT;
        // resident CTAs per SM: the descriptor's, else as many as shared memory allows (at
        // most 2 of 256 threads or 3 of 128: the register bound of the instances)
        int cps = (int)std::min<size_t>((smem_cap + 1024) / (smem + 1024), BM == 128 ? 2 : 3);
        if (v->ctas_per_sm > 0)
            cps = std::min(cps, v->ctas_per_sm);
        cps = std::max(cps, 1);
        long long grid = std::min<long long>(std::max<long long>(k.ntiles, 1), (long long)cps * sms);
        if (!cap_grid(grid, 1, v->max_ctas))
            return LC_ERR_INVALID_VARIANT;
        SimtGeom &g = r.g;
        g.grid = (int)grid;
        g.threads = BM / 8 * 16;
        g.smem = smem;
        g.TE = BM;
        g.ntiles = k.ntiles;
        g.nchunks = k.nblocks;
        return LC_OK;
    }
    if (v->engine == LC_ENGINE_WARP) {
        if (v->precision != LC_PREC_FP32 && v->precision != LC_PREC_FP64)
            return LC_ERR_INVALID_VARIANT;
        // registers hold F x N coefficients: FP32 N <= 32 (F <= 4); FP64 N <= 16 (F <= 4) or
        // N <= 32 with one operator
        if (N > 32 || F > 4 || (v->precision == LC_PREC_FP64 && N > 16 && F > 1))
            return LC_ERR_INVALID_VARIANT;
        const int per = 32 / N;
        if (v->tile_e <= 0 || v->tile_e % per != 0 || v->tile_e / per > 16)
            return LC_ERR_INVALID_VARIANT;
        if (v->unroll != 1 || v->prefetch_smem != 0 || v->stages != 1 || v->elems_per_thread != 1 ||
            v->split_i != 1)
            return LC_ERR_INVALID_VARIANT;
        r.warp_per = per;
        SimtGeom &g = r.g;
        g.threads = (v->tile_e / per) * 32;
        g.TE = v->tile_e;
        g.ntiles = (E + g.TE - 1) / g.TE;
        long long grid = g.ntiles;
        if (v->ctas_per_sm > 0)
            grid = std::min<long long>(grid, (long long)v->ctas_per_sm * sms);
        grid = std::max<long long>(grid, 1);
        if (!cap_grid(grid, 1, v->max_ctas))
            return LC_ERR_INVALID_VARIANT;
        g.grid = (int)grid;
        g.smem = 0;
        return LC_OK;
    }
    return LC_ERR_INVALID_VARIANT;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace lc

using namespace lc;

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *lc_status_string(lc_status s)
{
    switch (s) {
    case LC_OK: return "LC_OK";
    case LC_ERR_INVALID_ARGUMENT: return "LC_ERR_INVALID_ARGUMENT";
    case LC_ERR_UNSUPPORTED: return "LC_ERR_UNSUPPORTED";
    case LC_ERR_INVALID_VARIANT: return "LC_ERR_INVALID_VARIANT";
    case LC_ERR_ASSUMPTION: return "LC_ERR_ASSUMPTION";
    case LC_ERR_MISALIGNED: return "LC_ERR_MISALIGNED";
    case LC_ERR_BUFFER_TOO_SMALL: return "LC_ERR_BUFFER_TOO_SMALL";
    case LC_ERR_CUDA: return "LC_ERR_CUDA";
    case LC_ERR_TIMEOUT: return "LC_ERR_TIMEOUT";
    case LC_ERR_NO_DEVICE: return "LC_ERR_NO_DEVICE";
    case LC_ERR_NOT_FOUND: return "LC_ERR_NOT_FOUND";
    case LC_ERR_INDEX: return "LC_ERR_INDEX";
    }
    return "LC_ERR_UNKNOWN";
}

int lc_last_cuda_error(void) { return g_last_cuda_error; }

lc_status lc_kernel_create(const char *domain, const char *instructions, const char *assumptions,
                           lc_kernel **out)
{
    if (!domain || !instructions || !out)
        return LC_ERR_INVALID_ARGUMENT;
    Kernel K;
    std::string why;
    if (!parse_domain(domain, K, why))
        return LC_ERR_UNSUPPORTED;
    // the instruction forms, in turn: the contraction, the volume derivative with geometric factors
    const Kernel base = K;
    bool parsed = parse_instruction(instructions, K, why);
    if (!parsed) {
        K = base;
        parsed = parse_geo_instruction(instructions, K, why);
    }
    if (!parsed) {
        K = base;
        parsed = parse_lift_instruction(instructions, K, why);
    }
    if (!parsed) {
        K = base;
        parsed = parse_elementwise(instructions, K, why);
    }
    if (!parsed || !parse_assumptions(assumptions, K, why))
        return LC_ERR_UNSUPPORTED;
    K.domain_text = domain;
    K.insn_text = instructions;
    K.assumptions_text = assumptions ? assumptions : "";
    lc_kernel *h = new (std::nothrow) lc_kernel;
    if (!h)
        return LC_ERR_INVALID_ARGUMENT;
    h->k = std::move(K);
    *out = h;
    return LC_OK;
}

void lc_kernel_destroy(lc_kernel *k) { delete k; }

static void appendf(std::string &s, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s += buf;
}

lc_status lc_kernel_print(const lc_kernel *kh, const lc_variant *v, char *buf, size_t cap,
                          size_t *needed)
{
    if (!kh)
        return LC_ERR_INVALID_ARGUMENT;
    const Kernel &K = kh->k;
    const bool multi = !K.F_param.empty();
    const bool node = v && v->struct_size == sizeof(lc_variant) && v->layout == LC_LAYOUT_NODE_MAJOR;
    const char *ty = !v ? "<runtime>" : v->precision == LC_PREC_FP64 ? "float64" : "float32";
    const char *F = multi ? K.F_param.c_str() : "1";
    const char *E = K.E_param.c_str(), *N = K.N_param.c_str();
    std::string s;
    const char *rule = "------------------------------------------------------\n";
    const bool geo = K.kind == KIND_GEO;
    if (K.kind == KIND_LIFT) {
        const char *E = K.E_param.c_str(), *N = K.N_param.c_str(), *Nf = K.Nf_param.c_str(),
                   *Nfp = K.Nfp_param.c_str();
        s += rule;
        s += "KERNEL: dg_surface_lift\n";
        s += rule;
        s += "ARGUMENTS:\n";
        appendf(s, "%s: GlobalArg, type: float32, shape: (%s, %s, %s), dim_tags: (stride:%s*%s, stride:%s, stride:1)\n",
                K.d_name.c_str(), N, Nf, Nfp, Nf, Nfp, Nfp);
        appendf(s, "%s: GlobalArg, type: int32, shape: (%s, %s), dim_tags: (stride:%s, stride:1)\n",
                K.fmask_name.c_str(), Nf, Nfp, Nfp);
        appendf(s, "%s: GlobalArg, type: int32, shape: (%s, %s, %s), dim_tags: (stride:%s*%s, stride:%s, stride:1)\n",
                K.vmap_name.c_str(), E, Nf, Nfp, Nf, Nfp, Nfp);
        appendf(s, "%s: GlobalArg, type: float32, shape: (%s, %s), dim_tags: (stride:%s, stride:1)\n",
                K.s_name.c_str(), E, Nf, Nf);
        appendf(s, "%s: GlobalArg, type: float32, shape: (%s, %s), dim_tags: (stride:%s, stride:1)\n",
                K.u_name.c_str(), E, N, N);
        appendf(s, "%s: GlobalArg, type: float32, shape: (%s, %s), dim_tags: (stride:%s, stride:1), output\n",
                K.out_name.c_str(), E, N, N);
        s += rule;
        s += "DOMAINS:\n";
        appendf(s, "[%s, %s, %s, %s] -> { [%s, %s, %s, %s] : 0 <= %s < %s and 0 <= %s < %s and 0 <= %s < %s and "
                   "0 <= %s < %s }\n",
                E, N, Nf, Nfp, K.e_iname.c_str(), K.i_iname.c_str(), K.f_iname.c_str(), K.p_iname.c_str(),
                K.e_iname.c_str(), E, K.i_iname.c_str(), N, K.f_iname.c_str(), Nf, K.p_iname.c_str(), Nfp);
        if (!K.assumptions.empty()) {
            s += rule;
            appendf(s, "ASSUMPTIONS: %s\n", K.assumptions_text.c_str());
        }
        s += rule;
        s += "INSTRUCTIONS:\n";
        appendf(s, "[%s, %s] %s\n", K.e_iname.c_str(), K.i_iname.c_str(), K.insn_text.c_str());
        s += rule;
        if (needed)
            *needed = s.size() + 1;
        if (!buf || cap == 0)
            return LC_ERR_BUFFER_TOO_SMALL;
        size_t n = std::min(cap - 1, s.size());
        memcpy(buf, s.data(), n);
        buf[n] = 0;
        return n < s.size() ? LC_ERR_BUFFER_TOO_SMALL : LC_OK;
    }
    if (K.kind == KIND_ELEMENTWISE) {
        const bool two = K.inames.size() == 2;
        s += rule;
        s += "KERNEL: elementwise\n";
        s += rule;
        s += "ARGUMENTS:\n";
        for (size_t k = 0; k < K.ew.arrays.size(); ++k) {
            const EwArray &A = K.ew.arrays[k];
            std::string shape, tags;
            for (size_t q = 0; q < A.dims.size(); ++q) {
                shape += (q ? ", " : "") + K.bounds[A.dims[q]];
                tags += q ? ", stride:1" : (A.dims.size() == 2 ? "stride:" + K.bounds[A.dims[1]] : "stride:1");
            }
            appendf(s, "%s: GlobalArg, type: float32, shape: (%s), dim_tags: (%s)%s\n", A.name.c_str(), shape.c_str(),
                    tags.c_str(), k == 0 ? ", output" : "");
        }
        for (const auto &p : K.ew.params)
            appendf(s, "%s: ValueArg, type: float32\n", p.c_str());
        for (const auto &b : K.bounds)
            appendf(s, "%s: ValueArg, type: int64\n", b.c_str());
        s += rule;
        s += "DOMAINS:\n";
        std::string names, cons, params;
        for (size_t k = 0; k < K.inames.size(); ++k) {
            names += (k ? ", " : "") + K.inames[k];
            params += (k ? ", " : "") + K.bounds[k];
            cons += (k ? " and " : "") + std::string("0 <= ") + K.inames[k] + " < " + K.bounds[k];
        }
        appendf(s, "[%s] -> { [%s] : %s }\n", params.c_str(), names.c_str(), cons.c_str());
        if (!K.assumptions.empty()) {
            s += rule;
            appendf(s, "ASSUMPTIONS: %s\n", K.assumptions_text.c_str());
        }
        s += rule;
        s += "INSTRUCTIONS:\n";
        appendf(s, "[%s] %s\n", names.c_str(), K.insn_text.c_str());
        if (v && v->struct_size == sizeof(lc_variant)) {
            s += rule;
            s += "TRANSFORMATIONS:\n";
            const std::string &in = K.inames.back();
            const int tile = two ? 256 : 1024 * v->unroll;
            appendf(s, "split_iname(%s, %d): bulk tiles without guards, %s\n", in.c_str(), tile,
                    v->tail_free ? "no edge code (assumed divisible)" : "edge tile with a guard");
            if (two)
                appendf(s, "split_iname(%s, %d): edge code per bound and corner code for both\n", K.inames[0].c_str(),
                        4 * v->unroll);
            appendf(s, "tags: vec(%s) = %d, unr = %d, %d CTAs/SM\n", in.c_str(), v->elems_per_thread, v->unroll,
                    v->ctas_per_sm);
        }
        s += rule;
        if (needed)
            *needed = s.size() + 1;
        if (!buf || cap == 0)
            return LC_ERR_BUFFER_TOO_SMALL;
        size_t n = std::min(cap - 1, s.size());
        memcpy(buf, s.data(), n);
        buf[n] = 0;
        return n < s.size() ? LC_ERR_BUFFER_TOO_SMALL : LC_OK;
    }
    s += rule;
    s += geo ? "KERNEL: volume_derivative_with_geometric_factors\n" : "KERNEL: element_local_contraction\n";
    s += rule;
    s += "ARGUMENTS:\n";
    appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s, %s), dim_tags: (stride:%s*%s, stride:%s, stride:1)\n",
            K.d_name.c_str(), ty, F, N, N, N, N, N);
    if (geo) {
        if (node)
            appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s, %s), dim_tags: (stride:1, stride:%s*%s, stride:%s)\n",
                    K.g_name.c_str(), ty, E, F, F, F, E, E);
        else
            appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s, %s), dim_tags: (stride:%s*%s, stride:%s, stride:1)\n",
                    K.g_name.c_str(), ty, E, F, F, F, F, F);
    }
    if (multi)
        appendf(s, "%s: ValueArg, type: int32\n", F);
    appendf(s, "%s: ValueArg, type: int64\n%s: ValueArg, type: int32\n", E, N);
    if (node) {
        appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s, %s), dim_tags: (stride:%s*%s, stride:1, stride:%s)\n",
                K.out_name.c_str(), ty, F, E, N, N, E, E);
        appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s), dim_tags: (stride:1, stride:%s)\n",
                K.u_name.c_str(), ty, E, N, E);
    } else {
        appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s, %s), dim_tags: (stride:%s*%s, stride:%s, stride:1)\n",
                K.out_name.c_str(), ty, F, E, N, E, N, N);
        appendf(s, "%s: GlobalArg, type: %s, shape: (%s, %s), dim_tags: (stride:%s, stride:1)\n",
                K.u_name.c_str(), ty, E, N, N);
    }
    s += rule;
    s += "DOMAINS:\n";
    {
        std::string params, cons;
        std::set<std::string> seen;
        for (size_t k = 0; k < K.inames.size(); ++k) {
            if (!seen.count(K.bounds[k])) {
                if (!params.empty())
                    params += ", ";
                params += K.bounds[k];
                seen.insert(K.bounds[k]);
            }
            if (!cons.empty())
                cons += " and ";
            cons += "0 <= " + K.inames[k] + " < " + K.bounds[k];
        }
        std::string names;
        for (size_t k = 0; k < K.inames.size(); ++k)
            names += (k ? ", " : "") + K.inames[k];
        appendf(s, "[%s] -> { [%s] : %s }\n", params.c_str(), names.c_str(), cons.c_str());
    }
    if (!K.assumptions.empty()) {
        s += rule;
        appendf(s, "ASSUMPTIONS: %s\n", K.assumptions_text.c_str());
    }
    s += rule;
    s += "INSTRUCTIONS:\n";
    if (geo)
        appendf(s, "[%s, %s, %s] %s[%s, %s, %s] <- sum((%s, %s), %s[%s, %s, %s]*%s[%s, %s, %s]*%s[%s, %s])\n",
                K.d_iname.c_str(), K.e_iname.c_str(), K.i_iname.c_str(), K.out_name.c_str(), K.d_iname.c_str(),
                K.e_iname.c_str(), K.i_iname.c_str(), K.f_iname.c_str(), K.j_iname.c_str(), K.g_name.c_str(),
                K.e_iname.c_str(), K.d_iname.c_str(), K.f_iname.c_str(), K.d_name.c_str(), K.f_iname.c_str(),
                K.i_iname.c_str(), K.j_iname.c_str(), K.u_name.c_str(), K.e_iname.c_str(), K.j_iname.c_str());
    else if (multi)
        appendf(s, "[%s, %s, %s] %s[%s, %s, %s] <- sum(%s, %s[%s, %s, %s]*%s[%s, %s])\n",
                K.f_iname.c_str(), K.e_iname.c_str(), K.i_iname.c_str(), K.out_name.c_str(),
                K.f_iname.c_str(), K.e_iname.c_str(), K.i_iname.c_str(), K.j_iname.c_str(),
                K.d_name.c_str(), K.f_iname.c_str(), K.i_iname.c_str(), K.j_iname.c_str(),
                K.u_name.c_str(), K.e_iname.c_str(), K.j_iname.c_str());
    else
        appendf(s, "[%s, %s] %s[%s, %s] <- sum(%s, %s[%s, %s]*%s[%s, %s])\n", K.e_iname.c_str(),
                K.i_iname.c_str(), K.out_name.c_str(), K.e_iname.c_str(), K.i_iname.c_str(),
                K.j_iname.c_str(), K.d_name.c_str(), K.i_iname.c_str(), K.j_iname.c_str(),
                K.u_name.c_str(), K.e_iname.c_str(), K.j_iname.c_str());
    if (v && v->struct_size == sizeof(lc_variant)) {
        const char *eng = v->engine == LC_ENGINE_SIMT      ? "simt"
                          : v->engine == LC_ENGINE_TCGEN05 ? "tcgen05"
                          : v->engine == LC_ENGINE_KSPLIT  ? "ksplit"
                                                           : "warp";
        const char *prec[] = {"fp64", "fp32", "bf16", "bf16x3"};
        s += rule;
        s += "TRANSFORMATIONS:\n";
        appendf(s, "engine: %s, precision: %s, layout: %s-major\n", eng,
                (v->precision >= 0 && v->precision <= 3) ? prec[v->precision] : "?",
                node ? "node" : "element");
        const char *e = K.e_iname.c_str();
        appendf(s, "split_iname(%s, %d): %s = %s_inner + %d*%s_outer, %s_outer <= (%s + %d)/%d - 1\n", e,
                v->tile_e, e, e, v->tile_e, e, e, E, v->tile_e - 1, v->tile_e);
        if (v->tail_free)
            appendf(s, "  no guard: assumption %s mod %d = 0\n", E, v->tile_e);
        else
            appendf(s, "  guard: %s_inner + %d*%s_outer < %s on the last tile only\n", e, v->tile_e, e, E);
        appendf(s, "tags: %s_outer -> g.0 (persistent, %d CTAs/SM, at most %d CTAs; 0 = no bound), ilp(%s_inner) = %d, "
                   "ilp(%s) = %d, unr(%s) = %d\n",
                e, v->ctas_per_sm, v->max_ctas, e, v->elems_per_thread, K.i_iname.c_str(), v->split_i,
                K.j_iname.c_str(), v->unroll);
        appendf(s, "add_prefetch(%s): %s, stages: %d, output buffers: %d\n", K.u_name.c_str(),
                v->prefetch_smem ? "shared memory" : "none (global loads)", v->stages, v->out_buffers);
        if (v->engine == LC_ENGINE_TCGEN05)
            appendf(s, "rows per bulk store: %d (0 = planner's choice)\n", v->store_rows);
        if (v->engine == LC_ENGINE_KSPLIT)
            appendf(s, "split_iname(%s, %d): D^T chunks of %d rows fetched one chunk ahead\n", K.j_iname.c_str(),
                    v->unroll, v->unroll);
    }
    s += rule;
    if (needed)
        *needed = s.size() + 1;
    if (!buf || cap == 0)
        return LC_ERR_BUFFER_TOO_SMALL;
    size_t n = std::min(cap - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
    return n < s.size() ? LC_ERR_BUFFER_TOO_SMALL : LC_OK;
}

lc_status lc_variant_validate(const lc_kernel *kh, int64_t E, int32_t N, int32_t F, const lc_variant *v)
{
    if (!kh)
        return LC_ERR_INVALID_ARGUMENT;
    if (kh->k.kind == KIND_LIFT) {
        // E and N as for lc_lift; the descriptor: FP32 SIMT, element-major, grid fields,
        // staging buffers (stages 1 or 2), tile of 64 or 128 elements
        if (!v || v->struct_size != sizeof(lc_variant))
            return LC_ERR_INVALID_ARGUMENT;
        if (E < 0 || N < 1 || N > 128)
            return LC_ERR_INVALID_ARGUMENT;
        return (v->engine == LC_ENGINE_SIMT && v->precision == LC_PREC_FP32 && v->layout == LC_LAYOUT_ELEM_MAJOR &&
                v->ctas_per_sm >= 0 && v->ctas_per_sm <= 8 && v->max_ctas >= 0 && v->prefetch_smem >= 0 &&
                v->prefetch_smem <= 1 && v->stages >= 1 && v->stages <= 2 && (v->tile_e == 64 || v->tile_e == 128))
                   ? LC_OK
                   : LC_ERR_INVALID_VARIANT;
    }
    if (kh->k.kind == KIND_ELEMENTWISE) {
        // the extents of the first and second iname come as E and N; F must be 1
        const int64_t ext[2] = {E, N};
        int grid = 0;
        long long nt = 0;
        return F != 1 ? LC_ERR_INVALID_ARGUMENT : ew_validate(kh->k, v, ext, false, &grid, &nt);
    }
    Resolved r;
    return resolve(kh->k, E, N, F, v, r, false);
}

lc_status lc_variant_plan(const lc_kernel *kh, int64_t E, int32_t N, int32_t F, const lc_variant *v,
                          lc_plan *p)
{
    if (!kh || !p || p->struct_size != sizeof(lc_plan))
        return LC_ERR_INVALID_ARGUMENT;
    if (kh->k.kind == KIND_LIFT)
        return LC_ERR_UNSUPPORTED;  // the lift's plan needs Nf and Nfp (lc_lift)
    if (kh->k.kind == KIND_ELEMENTWISE) {
        const int64_t ext[2] = {E, N};
        int grid = 0;
        long long nt = 0;
        if (F != 1)
            return LC_ERR_INVALID_ARGUMENT;
        lc_status st = ew_validate(kh->k, v, ext, true, &grid, &nt);
        if (st == LC_ERR_NO_DEVICE)
            st = ew_validate(kh->k, v, ext, false, &grid, &nt);
        if (st != LC_OK)
            return st;
        lc_plan q;
        memset(&q, 0, sizeof q);
        q.struct_size = sizeof(lc_plan);
        q.grid = grid;
        q.threads = 256;
        q.tiles = nt;
        q.column_blocks = 1;
        *p = q;
        return LC_OK;
    }
    Resolved r;
    lc_status st = resolve(kh->k, E, N, F, v, r, true);
    if (st == LC_ERR_NO_DEVICE)
        st = resolve(kh->k, E, N, F, v, r, false);
    if (st != LC_OK)
        return st;
    lc_plan q;
    memset(&q, 0, sizeof q);
    q.struct_size = sizeof(lc_plan);
    if (r.engine == LC_ENGINE_TCGEN05) {
        const TcArgs &t = r.tc;
        const int nt = r.precision == LC_PREC_BF16X3 ? 3 : 1;
        q.grid = r.tc_grid;
        q.threads = tc_threads(t);
        q.smem_bytes = (int32_t)t.smem_bytes;
        q.tiles = t.ntiles;
        q.column_blocks = t.nblocks;
        q.ops_per_block = t.G;
        q.k_mma = t.Kt;
        q.k_block = t.KB;
        q.cols_per_op = t.Np;
        q.mma_n = t.CBp;
        q.stacked = t.stack;
        q.a_buffers = t.abufs;
        q.out_slots = r.layout == LC_LAYOUT_ELEM_MAJOR ? t.obufs : 0;
        q.store_rows = r.layout == LC_LAYOUT_ELEM_MAJOR ? 32 * t.store_quarters : 0;
        q.mma_per_tile = (nt == 1 ? 1 : (t.stack ? 5 : 6)) * (q.k_mma / 16);
        q.a_in_tmem = t.a_tmem;
        q.tmem_cols = t.tmem_alloc;
    } else {
        q.grid = r.g.grid;
        q.threads = r.g.threads;
        q.smem_bytes = (int32_t)r.g.smem;
        q.tiles = r.g.ntiles;
        q.column_blocks = (r.engine == LC_ENGINE_SIMT || r.engine == LC_ENGINE_KSPLIT) ? r.g.nchunks : 1;
        q.ops_per_block = r.engine == LC_ENGINE_SIMT ? (r.g.isplit ? 0 : r.g.G) : F;
    }
    *p = q;
    return LC_OK;
}

lc_status lc_variant_default(const lc_kernel *kh, int64_t E, int32_t N, int32_t F, int32_t layout,
                             int32_t precision, lc_variant *v)
{
    if (!kh || !v)
        return LC_ERR_INVALID_ARGUMENT;
    lc_variant d;
    memset(&d, 0, sizeof d);
    d.struct_size = sizeof(lc_variant);
    if (kh->k.kind == KIND_LIFT) {
        if (precision != LC_PREC_FP32 || layout != LC_LAYOUT_ELEM_MAJOR)
            return LC_ERR_UNSUPPORTED;
        // one staging buffer, three CTAs per SM (E = 2^21, degree 4: 0.60 ms, against 0.72 ms
        // with two buffers, where only two CTAs fit)
        d.engine = LC_ENGINE_SIMT;
        d.precision = LC_PREC_FP32;
        d.tile_e = 64;
        d.elems_per_thread = 4;
        d.split_i = 4;
        d.unroll = 4;
        d.prefetch_smem = 1;
        d.stages = 1;
        d.ctas_per_sm = 3;
        *v = d;
        return LC_OK;
    }
    if (kh->k.kind == KIND_ELEMENTWISE) {
        // 16-byte vectors, four per thread and tile, four CTAs per SM; FP32
        if (precision != LC_PREC_FP32 || layout != LC_LAYOUT_ELEM_MAJOR)
            return LC_ERR_UNSUPPORTED;
        d.engine = LC_ENGINE_SIMT;
        d.precision = LC_PREC_FP32;
        d.unroll = 4;
        d.elems_per_thread = 4;
        d.stages = 1;
        d.ctas_per_sm = 4;
        *v = d;
        return LC_OK;
    }
    d.layout = layout;
    d.precision = precision;
    d.unroll = 4;
    d.stages = 1;
    d.prefetch_smem = 1;
    d.ctas_per_sm = 0;
    if (precision == LC_PREC_FP64) {
        d.engine = LC_ENGINE_SIMT;
        d.elems_per_thread = 4;
        d.split_i = 4;
        d.tile_e = 64;
        d.stages = 2;
    } else if (precision == LC_PREC_FP32) {
        if (precision == LC_PREC_FP32 && N >= 96) {
            // large N: the K-split kernel (D^T streamed in chunks) measured faster than the
            // SIMT kernel holding all of D^T (N = 120: 0.69 against 0.86 ms; N = 165: 2.6
            // against 3.6 ms)
            lc_variant k = d;
            k.engine = LC_ENGINE_KSPLIT;
            k.tile_e = 128;
            k.elems_per_thread = 8;
            k.split_i = 8;
            k.unroll = 8;
            k.prefetch_smem = 1;
            k.stages = 1;
            if (lc_variant_validate(kh, E, N, F, &k) == LC_OK) {
                *v = k;
                return LC_OK;
            }
        }
        if (N <= 12) {
            // small N: the warp engine (32 / N elements a warp, D rows in registers, u values
            // passed by shuffles); measured at N = 4, E = 360273: 12 us against 32 us for
            // the SIMT tiles
            lc_variant w = d;
            w.engine = LC_ENGINE_WARP;
            w.tile_e = (32 / N) * 8;
            w.elems_per_thread = 1;
            w.split_i = 1;
            w.unroll = 1;
            w.prefetch_smem = 0;
            w.stages = 1;
            w.ctas_per_sm = 4;
            if (lc_variant_validate(kh, E, N, F, &w) == LC_OK) {
                *v = w;
                return LC_OK;
            }
        }
        // SIMT tiles, two CTAs per SM, the u tile staged by bulk copies two tiles ahead; the
        // fastest measured per layout and node count (autotuner, N = 20 .. 84, F = 2 .. 4):
        // element-major 4 x 8 register blocks with j unrolled 4 times, 64-element tiles up to
        // N = 40 and 32 above (N = 56: 0.58 ms against 1.00 ms for 128-element tiles of 8 x 8
        // blocks); node-major without unrolling (N = 56: 0.57 against 0.77 ms unrolled)
        d.engine = LC_ENGINE_SIMT;
        d.ctas_per_sm = 2;
        d.prefetch_smem = 1;
        d.stages = 2;
        if (layout == LC_LAYOUT_ELEM_MAJOR) {
            d.elems_per_thread = 4;
            d.split_i = 8;
            d.tile_e = N <= 40 ? 64 : 32;
            d.unroll = 4;
        } else if (N <= 24) {
            d.elems_per_thread = 8;
            d.split_i = 4;
            d.tile_e = 128;
            d.unroll = 4;
        } else if (N <= 40) {
            d.elems_per_thread = 8;
            d.split_i = 8;
            d.tile_e = 128;
            d.unroll = 1;
        } else {
            d.elems_per_thread = 4;
            d.split_i = 8;
            d.tile_e = N <= 72 ? 64 : 32;
            d.unroll = 1;
        }
    } else {
        d.engine = LC_ENGINE_TCGEN05;
        d.tile_e = 128;
        d.split_i = 0;
        d.unroll = 4;
        // BF16X3: three epilogue and conversion threads per row with the stage released early
        // (element-major), two with two stages (node-major): the fastest measured at N = 35
        // 64-wide K-blocks first: a tcgen05.mma reading 128-byte swizzled rows costs the
        // fewest cycles; then the narrowest blocks that cover K (least shared memory).
        // BF16X3: the A terms in shared memory first (the stacked order), one stage first (two
        // stages leave room for one output slot only); BF16: the planner's placement, two stages.
        const bool x3 = precision == LC_PREC_BF16X3;
        lc_status st = LC_ERR_INVALID_VARIANT;
        const bool x3node = x3 && layout == LC_LAYOUT_NODE_MAJOR;
        if (x3) {
            d.unroll = x3node ? 2 : 3;
            d.prefetch_smem = x3node ? 1 : 2;
        }
        for (int aop : {x3 ? 1 : 0})
            for (int kbw : {64, 1})
                for (int stg : {x3 && !x3node ? 1 : 2, x3 && !x3node ? 2 : 3, 1}) {
                    if (st == LC_OK)
                        break;
                    d.a_operand = aop;
                    d.elems_per_thread = kbw;
                    d.stages = stg;
                    st = lc_variant_validate(kh, E, N, F, &d);
                    if (st != LC_OK && st != LC_ERR_INVALID_VARIANT)
                        return st;
                }
        if (st != LC_OK && x3) {
            // no shared-memory plan for the three A terms (N of about 100 and more): the
            // planner's placement (tensor memory), one operator per column block, 32-row
            // stores; measured at N = 120, E = 310977: 0.44 ms against 0.69 ms for the K-split
            // FP32 kernel (node-major 0.65 against 0.89 ms)
            d.a_operand = 0;
            d.split_i = 1;
            d.unroll = 3;
            d.prefetch_smem = 1;
            d.stages = 1;
            d.store_rows = layout == LC_LAYOUT_ELEM_MAJOR ? 32 : 0;
            for (int kbw : {64, 1}) {
                d.elems_per_thread = kbw;
                st = lc_variant_validate(kh, E, N, F, &d);
                if (st == LC_OK || st != LC_ERR_INVALID_VARIANT)
                    break;
            }
        }
        if (st == LC_OK) {
            *v = d;
            return LC_OK;
        }
        if (st != LC_ERR_INVALID_VARIANT)
            return st;
        if (kh->k.kind == KIND_GEO)
            return LC_ERR_UNSUPPORTED;  // the volume derivative runs on the tensor cores only
        // no tensor-core plan fits (large N): FP32, whose error is below both
        // reduced-precision bounds
        return lc_variant_default(kh, E, N, F, layout, LC_PREC_FP32, v);
    }
    // shrink the tile (then the register block) until the shared-memory plan fits
    const lc_variant d0 = d;
    for (int attempt = 0; attempt < 2; ++attempt) {
        while (d.tile_e > d.elems_per_thread && lc_variant_validate(kh, E, N, F, &d) == LC_ERR_INVALID_VARIANT)
            d.tile_e /= 2;
        if (lc_variant_validate(kh, E, N, F, &d) != LC_ERR_INVALID_VARIANT)
            break;
        d = d0;
        d.elems_per_thread = precision == LC_PREC_FP64 ? 2 : 4;
        d.split_i = precision == LC_PREC_FP64 ? 2 : 4;
    }
    lc_status st = lc_variant_validate(kh, E, N, F, &d);
    if (st != LC_OK)
        return st;
    *v = d;
    return LC_OK;
}

lc_status lc_contract(const lc_kernel *kh, const lc_variant *v, const void *D, const void *u, void *out,
                      int64_t E, int32_t N, int32_t F, void *stream)
{
    if (!kh || !v)
        return LC_ERR_INVALID_ARGUMENT;
    if (kh->k.kind != KIND_CONTRACT)
        return LC_ERR_UNSUPPORTED;
    // an empty batch may come with null u / out (zero-size allocations)
    if (!D || (E > 0 && (!u || !out)))
        return LC_ERR_INVALID_ARGUMENT;
    if (!aligned16(D) || !aligned16(u) || !aligned16(out))
        return LC_ERR_MISALIGNED;
    Resolved r;
    lc_status st = resolve(kh->k, E, N, F, v, r, true);
    if (st != LC_OK)
        return st;
    const size_t es = v->precision == LC_PREC_FP64 ? 8 : 4;
    {
        // out must not overlap its inputs
        uintptr_t o0 = (uintptr_t)out, o1 = o0 + (size_t)F * E * N * es;
        uintptr_t u0 = (uintptr_t)u, u1 = u0 + (size_t)E * N * es;
        uintptr_t d0 = (uintptr_t)D, d1 = d0 + (size_t)F * N * N * es;
        if ((o0 < u1 && u0 < o1) || (o0 < d1 && d0 < o1))
            return LC_ERR_INVALID_ARGUMENT;
    }
    int major = 0, minor = 0;
    if (current_cc(&major, &minor) != 0 || major != 10 || minor != 3)
        return LC_ERR_NO_DEVICE;
    if (E == 0)
        return LC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (r.engine == LC_ENGINE_SIMT) {
        SimtArgs a;
        a.D = D;
        a.u = u;
        a.out = out;
        a.E = E;
        a.N = N;
        a.F = F;
        a.C = F * N;
        a.TE = r.g.TE;
        a.EG = r.g.EG;
        a.CG = r.g.CG;
        a.CW = r.g.CW;
        a.nchunks = r.g.nchunks;
        a.G = r.g.G;
        a.isplit = r.g.isplit;
        a.WC = r.g.WC;
        a.stages = r.g.stages;
        a.bulk = r.g.bulk;
        a.bulk_store = r.g.bulk_store;
        a.ntiles = r.g.ntiles;
        a.tail_free = r.tail_free;
        a.err = error_word();
        const bool node = r.layout == LC_LAYOUT_NODE_MAJOR;
        if (r.precision == LC_PREC_FP32)
            return node ? simt_launch_f32_node(a, r.g, r.unroll, r.prefetch, s)
                        : simt_launch_f32_elem(a, r.g, r.unroll, r.prefetch, s);
        return node ? simt_launch_f64_node(a, r.g, r.unroll, r.prefetch, s)
                    : simt_launch_f64_elem(a, r.g, r.unroll, r.prefetch, s);
    }
    if (r.engine == LC_ENGINE_TCGEN05) {
        TcArgs a = r.tc;
        a.D = static_cast<const float *>(D);
        a.u = static_cast<const float *>(u);
        a.out = static_cast<float *>(out);
        a.err = error_word();
        return tc_launch(a, r.layout, r.precision == LC_PREC_BF16X3 ? 3 : 1, r.tc_grid, s);
    }
    if (r.engine == LC_ENGINE_KSPLIT) {
        KsArgs a = r.ks;
        a.D = static_cast<const float *>(D);
        a.u = static_cast<const float *>(u);
        a.out = static_cast<float *>(out);
        return ks_launch(a, r.layout, r.ks_bm, r.ks_bk, r.g.grid, s);
    }
    if (r.engine == LC_ENGINE_WARP) {
        WarpArgs a;
        a.D = D;
        a.u = u;
        a.out = out;
        a.E = E;
        a.N = N;
        a.F = F;
        a.per_warp = r.warp_per;
        a.ngroups = (E + r.warp_per - 1) / r.warp_per;
        a.tail_free = r.tail_free;
        return warp_launch(a, r.layout, r.precision == LC_PREC_FP64, r.g.grid, r.g.threads, s);
    }
    return LC_ERR_INVALID_VARIANT;
}

lc_status lc_contract_geo(const lc_kernel *kh, const lc_variant *v, const void *D, const void *u, const void *r,
                          void *out, int64_t E, int32_t N, int32_t F, void *stream)
{
    if (!kh || !v)
        return LC_ERR_INVALID_ARGUMENT;
    if (kh->k.kind != KIND_GEO)
        return LC_ERR_UNSUPPORTED;
    if (!D || (E > 0 && (!u || !out || !r)))
        return LC_ERR_INVALID_ARGUMENT;
    if (!aligned16(D) || !aligned16(u) || !aligned16(out) || !aligned16(r))
        return LC_ERR_MISALIGNED;
    Resolved rs;
    lc_status st = resolve(kh->k, E, N, F, v, rs, true);
    if (st != LC_OK)
        return st;
    {
        // out must not overlap its inputs
        const uintptr_t o0 = (uintptr_t)out, o1 = o0 + (size_t)F * E * N * 4;
        const uintptr_t in[3][2] = {{(uintptr_t)u, (uintptr_t)u + (size_t)E * N * 4},
                                    {(uintptr_t)D, (uintptr_t)D + (size_t)F * N * N * 4},
                                    {(uintptr_t)r, (uintptr_t)r + (size_t)E * F * F * 4}};
        for (auto &x : in)
            if (o0 < x[1] && x[0] < o1)
                return LC_ERR_INVALID_ARGUMENT;
    }
    int major = 0, minor = 0;
    if (current_cc(&major, &minor) != 0 || major != 10 || minor != 3)
        return LC_ERR_NO_DEVICE;
    if (E == 0)
        return LC_OK;
    TcArgs a = rs.tc;
    a.D = static_cast<const float *>(D);
    a.u = static_cast<const float *>(u);
    a.out = static_cast<float *>(out);
    a.r = static_cast<const float *>(r);
    a.err = error_word();
    return tc_geo_launch(a, rs.layout, rs.precision == LC_PREC_BF16X3 ? 3 : 1, rs.tc_grid, (cudaStream_t)stream);
}

namespace lc {

// Copy streams of the host-array entry point, one per direction and device, created on
// first use and kept for the life of the process.  (A second stream per direction, with
// chunks alternating, measured no faster: the host link, not one copy engine, is the limit.)
static constexpr int kCopyStreams = 2;  // in, out
static std::mutex g_copy_mu;
static std::map<int, std::array<cudaStream_t, kCopyStreams>> g_copy_streams;

static lc_status copy_streams(cudaStream_t *cs)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e);
    std::lock_guard<std::mutex> lk(g_copy_mu);
    auto it = g_copy_streams.find(dev);
    if (it == g_copy_streams.end()) {
        std::array<cudaStream_t, kCopyStreams> a{};
        for (auto &x : a)
            if (e == cudaSuccess)
                e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return cuda_fail(e);
        it = g_copy_streams.emplace(dev, a).first;
    }
    for (int i = 0; i < kCopyStreams; ++i)
        cs[i] = it->second[i];
    return LC_OK;
}

}  // namespace lc

lc_status lc_contract_host(const lc_kernel *kh, const lc_variant *v, const void *D_host, const void *u_host,
                           void *out_host, int64_t E, int32_t N, int32_t F, void *D_dev, void *u_dev,
                           void *out_dev, void *stream)
{
    if (!kh || !v || !D_host || !u_host || !out_host || !D_dev || !u_dev || !out_dev)
        return LC_ERR_INVALID_ARGUMENT;
    if (v->struct_size != sizeof(lc_variant) || E < 0 || N < 1 || F < 1)
        return LC_ERR_INVALID_ARGUMENT;
    Resolved r;
    lc_status st = resolve(kh->k, E, N, F, v, r, true);
    if (st != LC_OK)
        return st;
    if (E == 0)
        return LC_OK;
    const size_t es = v->precision == LC_PREC_FP64 ? 8 : 4;
    const bool node = v->layout == LC_LAYOUT_NODE_MAJOR;
    cudaStream_t s = (cudaStream_t)stream;

    // Element chunks (whole 128-element tiles, at least 2^16 elements, at most 8): the
    // copy of chunk c+1 in, the contraction of chunk c and the copy of chunk c-1 out run
    // at the same time (two copy streams and the caller's stream, ordered by events).
    // Each chunk's u and out are packed in the caller's device buffers at its element
    // offset, so chunks never share device memory.
    long long chunk = E;
    int nchunks = 1;
    {
        const long long want = std::min<long long>(8, E >> 16);
        if (want > 1) {
            const long long c = ((E + want - 1) / want + 127) / 128 * 128;
            Resolved r1, r2;
            const long long last = E - (long long)((E - 1) / c) * c;
            if (resolve(kh->k, c, N, F, v, r1, true) == LC_OK && resolve(kh->k, last, N, F, v, r2, true) == LC_OK) {
                chunk = c;
                nchunks = (int)((E + c - 1) / c);
            }
        }
    }
    cudaStream_t cs[lc::kCopyStreams];
    st = lc::copy_streams(cs);
    if (st != LC_OK)
        return st;
    std::vector<cudaEvent_t> ev(2 * (size_t)nchunks + 2, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &x : ev)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    auto cleanup = [&]() {
        for (auto &x : ev)
            if (x)
                cudaEventDestroy(x);  // released once the recorded work completes
    };
    auto fail = [&](cudaError_t err) {
        cleanup();
        return lc::cuda_fail(err);
    };
    if (e != cudaSuccess)
        return fail(e);
    cudaEvent_t ev_start = ev[2 * nchunks], ev_done = ev[2 * nchunks + 1];
    // nothing starts before the work already queued on the caller's stream
    e = cudaEventRecord(ev_start, s);
    for (int i = 0; i < lc::kCopyStreams; ++i)
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(cs[i], ev_start, 0);
    if (e == cudaSuccess)  // before chunk 0's input on the same stream; every contraction follows chunk 0's
        e = cudaMemcpyAsync(D_dev, D_host, (size_t)F * N * N * es, cudaMemcpyHostToDevice, cs[0]);
    if (e != cudaSuccess)
        return fail(e);
    const char *uh = static_cast<const char *>(u_host);
    char *ud = static_cast<char *>(u_dev), *oh = static_cast<char *>(out_host), *od = static_cast<char *>(out_dev);
    for (int c = 0; c < nchunks; ++c) {
        const long long e0 = (long long)c * chunk, ec = std::min(chunk, E - e0);
        char *u_c = ud + (size_t)e0 * N * es;      // packed chunk input  (elem: [ec][N], node: [N][ec])
        char *o_c = od + (size_t)e0 * F * N * es;  // packed chunk output (elem: [F][ec][N], node: [F][N][ec])
        cudaEvent_t ev_in = ev[2 * c], ev_comp = ev[2 * c + 1];
        cudaStream_t s_in = cs[0], s_out = cs[1];
        if (node)
            e = cudaMemcpy2DAsync(u_c, (size_t)ec * es, uh + (size_t)e0 * es, (size_t)E * es, (size_t)ec * es, N,
                                  cudaMemcpyHostToDevice, s_in);
        else
            e = cudaMemcpyAsync(u_c, uh + (size_t)e0 * N * es, (size_t)ec * N * es, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess)
            e = cudaEventRecord(ev_in, s_in);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, ev_in, 0);
        if (e != cudaSuccess)
            return fail(e);
        st = lc_contract(kh, v, D_dev, u_c, o_c, ec, N, F, stream);
        if (st != LC_OK) {
            cleanup();
            return st;
        }
        e = cudaEventRecord(ev_comp, s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s_out, ev_comp, 0);
        if (e == cudaSuccess) {
            if (node)  // F*N rows of ec values
                e = cudaMemcpy2DAsync(oh + (size_t)e0 * es, (size_t)E * es, o_c, (size_t)ec * es, (size_t)ec * es,
                                      (size_t)F * N, cudaMemcpyDeviceToHost, s_out);
            else  // F rows of ec*N values
                e = cudaMemcpy2DAsync(oh + (size_t)e0 * N * es, (size_t)E * N * es, o_c, (size_t)ec * N * es,
                                      (size_t)ec * N * es, F, cudaMemcpyDeviceToHost, s_out);
        }
        if (e != cudaSuccess)
            return fail(e);
    }
    // the caller's stream resumes after the last copy out
    e = cudaEventRecord(ev_done, cs[1]);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s, ev_done, 0);
    if (e != cudaSuccess)
        return fail(e);
    cleanup();
    return LC_OK;
}

// ------------------------------------------------------------------ grouped launch

namespace lc {
// One plain K-split launch: a group of a tensor-core grouped plan without a tensor-core plan,
// or a large-N group of an FP32 grouped plan.
struct KsLaunch {
    KsArgs a;
    int grid, bm, bk, group;
};

// One plain tensor-core launch: a group of a tensor-core grouped plan whose plan needs the A
// terms in tensor memory (no shared-memory plan fits), which the grouped kernel does not take.
struct TcLaunch {
    TcArgs a;
    int layout, nterms, grid, group;
};

}  // namespace lc

struct lc_grouped_plan {
    // SIMT part (every group of a SIMT plan; the groups without a tensor plan of a tensor plan)
    void *fn = nullptr;
    GroupedArgs args{};
    int grid = 0, threads = 0;
    size_t smem = 0;
    // tensor-core part
    void *fn_tc = nullptr;
    lc::TcGroupedParams tcp{};
    int grid_tc = 0, threads_tc = 0;
    size_t smem_tc = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int ngroups = 0, nsegs = 0;
    std::vector<lc_variant> group_variant;  // the descriptor serving each group
    std::vector<lc::KsLaunch> ks;           // K-split launches (after the tensor-core one)
    std::vector<lc::TcLaunch> tcl;          // single-group tensor-core launches (after the K-split ones)
    int layout = 0;
};

namespace lc {

struct GroupedPlanHost {
    std::vector<SimtArgs> groups;
    std::vector<GroupSeg> segs;
    std::vector<int> cta_seg;
    size_t smem = 0, bytes = 0;
    size_t off_groups = 0, off_segs = 0, off_cta = 0;
    int grid = 0, threads = 256;
};

static lc_status grouped_plan_host(const Kernel &K, const lc_variant *v, const lc_group *groups, int ng,
                                   GroupedPlanHost &P)
{
    if (!v || v->struct_size != sizeof(lc_variant) || !groups || ng <= 0)
        return LC_ERR_INVALID_ARGUMENT;
    if (v->engine != LC_ENGINE_SIMT || v->precision != LC_PREC_FP32 || v->tail_free)
        return LC_ERR_INVALID_VARIANT;
    if (!(v->unroll == 1 || v->unroll == 4))
        return LC_ERR_INVALID_VARIANT;
    const int sms = sm_count();
    if (sms <= 0)
        return LC_ERR_NO_DEVICE;
    // CTA size: the most threads the register block allows (the same bound as the plain kernel)
    P.threads = v->elems_per_thread * v->split_i >= 64 ? 256 : 512;
    const int T = P.threads;
    std::vector<double> tile_cost(ng);
    P.groups.resize(ng);
    P.smem = 0;
    for (int gi = 0; gi < ng; ++gi) {
        const lc_group &G = groups[gi];
        if (!G.D_dev || (G.E > 0 && (!G.u_dev || !G.out_dev)))
            return LC_ERR_INVALID_ARGUMENT;
        if (!aligned16(G.D_dev) || !aligned16(G.u_dev) || !aligned16(G.out_dev))
            return LC_ERR_MISALIGNED;
        // tile of TE = EG * RE elements within T threads: the most active threads, then the
        // fewest padded columns, then the largest tile (fewer, longer bulk copies per tile).
        // Node-major also counts column blocks: each one reads the u tile again with plain
        // loads (the bulk engine needs 16-byte aligned rows of u), which costs more than
        // idle threads do.
        Resolved best;
        double best_key = 0;
        bool have = false;
        for (int eg = 4; eg <= T; eg *= 2) {
            lc_variant vg = *v;
            vg.tile_e = eg * v->elems_per_thread;
            vg.ctas_per_sm = 0;
            Resolved r;
            if (resolve(K, G.E, G.N, G.F, &vg, r, true, T) != LC_OK)
                continue;
            const double idle = (double)(T - r.g.threads) / T;
            const double pad = (double)(r.g.nchunks * (long long)r.g.CW) / ((double)G.F * G.N) - 1.0;
            const bool nodel = v->layout == LC_LAYOUT_NODE_MAJOR;
            // node-major: the tile the autotuner measured fastest for the plain SIMT kernel at
            // this N (lc_variant_default) comes first (grouped, full-size uneven batching: 7.9
            // against 8.5 ms; element-major kept the weighted sum: 6.2 against 6.6 ms); the
            // weighted sum orders the rest
            const int pref = nodel ? (G.N <= 40 ? 128 : G.N <= 72 ? 64 : 32) : 0;
            const double key = (vg.tile_e == pref ? -100.0 : 0.0) + idle * (nodel ? 0.25 : 4.0) + pad +
                               (nodel ? 0.5 * (r.g.nchunks - 1) : 0.0) - 0.05 * std::log2((double)vg.tile_e);
            if (!have || key < best_key) {
                best_key = key;
                best = r;
                have = true;
            }
        }
        if (!have)
            return LC_ERR_INVALID_VARIANT;
        SimtArgs a;
        memset(&a, 0, sizeof a);
        a.D = G.D_dev;
        a.u = G.u_dev;
        a.out = G.out_dev;
        a.E = G.E;
        a.N = G.N;
        a.F = G.F;
        a.C = G.F * G.N;
        a.TE = best.g.TE;
        a.EG = best.g.EG;
        a.CG = best.g.CG;
        a.CW = best.g.CW;
        a.nchunks = best.g.nchunks;
        a.G = best.g.G;
        a.isplit = best.g.isplit;
        a.WC = best.g.WC;
        a.stages = best.g.stages;
        a.bulk = best.g.bulk;
        a.bulk_store = best.g.bulk_store;
        a.ntiles = best.g.ntiles;
        a.tail_free = 0;
        P.groups[gi] = a;
        P.smem = std::max(P.smem, best.g.smem);
        // estimated seconds per item: FMA pipe (FP32, padded columns) vs HBM
        const double flops = 2.0 * a.TE * (double)G.N * a.CW;
        const double bytes = 4.0 * a.TE * ((double)G.N + (a.isplit ? a.isplit : (double)a.G * G.N));
        tile_cost[gi] = std::max(flops / (sms * 128 * 2 * 1.9e9), bytes / 6.8e12) + 2e-7 / sms;
    }
    // units: (group, column block) with its tiles and cost per tile
    struct Unit {
        int g, chunk;
        long long tiles;
        double cost;
    };
    std::vector<Unit> units;
    double total = 0;
    long long total_items = 0;
    for (int gi = 0; gi < ng; ++gi) {
        const long long tiles_g = groups[gi].E > 0 ? P.groups[gi].ntiles : 0;
        for (int ch = 0; ch < P.groups[gi].nchunks && tiles_g > 0; ++ch) {
            units.push_back({gi, ch, tiles_g, tile_cost[gi]});
            total += tiles_g * tile_cost[gi];
            total_items += tiles_g;
        }
    }
    const int per_sm = v->ctas_per_sm > 0 ? v->ctas_per_sm : 2;
    long long cap = (long long)sms * per_sm;
    if (v->max_ctas > 0)
        cap = std::min<long long>(cap, v->max_ctas);
    P.grid = (int)std::max<long long>(1, std::min<long long>(cap, total_items));
    const double budget = total / P.grid;
    // CTAs per big unit (worth >= 1 CTA), the rest for the small units
    std::vector<int> alloc(units.size(), 0);
    double small_work = 0;
    int nbig = 0;
    for (size_t q = 0; q < units.size(); ++q) {
        const double w = units[q].tiles * units[q].cost / budget;
        if (w >= 1.0) {
            alloc[q] = (int)std::min<long long>((long long)w, units[q].tiles);
            ++nbig;
        } else {
            small_work += w;
        }
    }
    const int small_ctas = small_work > 0 ? std::max(1, (int)std::ceil(small_work)) : 0;
    auto used = [&]() {
        long long sum = small_ctas;
        for (int x : alloc)
            sum += x;
        return sum;
    };
    while (used() > P.grid) {  // shrink the unit with the most CTAs
        size_t m = 0;
        for (size_t q = 1; q < alloc.size(); ++q)
            if (alloc[q] > alloc[m])
                m = q;
        if (alloc[m] <= 1)
            break;
        --alloc[m];
    }
    while (nbig > 0 && used() < P.grid) {  // give spare CTAs to the most loaded big unit
        size_t m = alloc.size();
        double worst = -1;
        for (size_t q = 0; q < alloc.size(); ++q) {
            if (alloc[q] == 0 || alloc[q] >= units[q].tiles)
                continue;
            const double load = units[q].tiles * units[q].cost / alloc[q];
            if (load > worst) {
                worst = load;
                m = q;
            }
        }
        if (m == alloc.size())
            break;
        ++alloc[m];
    }
    P.grid = (int)std::max<long long>(1, used());
    std::vector<std::vector<GroupSeg>> per_cta(P.grid);
    int b = 0;
    for (size_t q = 0; q < units.size(); ++q) {
        if (alloc[q] == 0)
            continue;
        const int n = alloc[q];
        for (int r = 0; r < n; ++r) {
            GroupSeg sg;
            sg.group = units[q].g;
            sg.chunk = units[q].chunk;
            sg.first = r;
            sg.step = n;
            sg.count = (units[q].tiles - r + n - 1) / n;
            per_cta[b + r].push_back(sg);
        }
        b += n;
    }
    // small units: whole, onto the least loaded of the remaining CTAs
    std::vector<double> load(P.grid, 0.0);
    for (size_t q = 0; q < units.size(); ++q) {
        if (alloc[q] != 0)
            continue;
        int best = b;
        for (int c = b; c < P.grid; ++c)
            if (load[c] < load[best])
                best = c;
        if (best >= P.grid)
            best = P.grid - 1;
        GroupSeg sg;
        sg.group = units[q].g;
        sg.chunk = units[q].chunk;
        sg.first = 0;
        sg.step = 1;
        sg.count = units[q].tiles;
        per_cta[best].push_back(sg);
        load[best] += units[q].tiles * units[q].cost;
    }
    P.segs.clear();
    P.cta_seg.assign(P.grid + 1, 0);
    for (int c = 0; c < P.grid; ++c) {
        P.cta_seg[c] = (int)P.segs.size();
        for (const GroupSeg &sg : per_cta[c])
            P.segs.push_back(sg);
    }
    P.cta_seg[P.grid] = (int)P.segs.size();
    auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
    P.off_groups = 0;
    P.off_segs = up16(sizeof(SimtArgs) * ng);
    P.off_cta = P.off_segs + up16(sizeof(GroupSeg) * P.segs.size());
    P.bytes = P.off_cta + up16(sizeof(int) * (P.grid + 1));
    return LC_OK;
}

// Tensor-core part of a grouped plan: the groups with a tensor-core plan for the variant
// (their indices in `tc_groups`, the rest in `simt_groups`), one (group, column block) unit per
// CTA set, CTAs handed out so that the slowest unit's estimated time is the least, at most one
// CTA per SM.
struct GroupedPlanTc {
    TcGroupedParams P{};
    std::vector<lc_variant> gv;  // per group: the tensor-core variant serving it
    std::vector<int4> map;
    int grid = 0, threads = 0, nterms = 1;
    size_t smem = 0;
    std::vector<int> tc_groups, simt_groups;
};

static lc_status grouped_plan_tc(const Kernel &K, const lc_variant *v, const lc_group *groups, int ng,
                                 GroupedPlanTc &T)
{
    if (ng > kTcMaxGroups)
        return LC_ERR_INVALID_ARGUMENT;
    for (int gi = 0; gi < ng; ++gi) {
        const lc_group &G = groups[gi];
        if (!G.D_dev || (G.E > 0 && (!G.u_dev || !G.out_dev)))
            return LC_ERR_INVALID_ARGUMENT;
        if (!aligned16(G.D_dev) || !aligned16(G.u_dev) || !aligned16(G.out_dev))
            return LC_ERR_MISALIGNED;
    }
    const int sms = sm_count();
    if (sms <= 0)
        return LC_ERR_NO_DEVICE;
    T.nterms = v->precision == LC_PREC_BF16X3 ? 3 : 1;
    T.gv.assign(ng, *v);
    struct Unit {
        int g, blk;
        long long tiles;
        double cost;  // estimated seconds per tile
    };
    std::vector<Unit> units;
    for (int gi = 0; gi < ng; ++gi) {
        const lc_group &G = groups[gi];
        // the variant as given, else the first of: one stage, the other K-block width
        // (1 <-> 64), 32-row stores (element-major), that has a plan; the CTA size stays
        Resolved r;
        lc_status rs = LC_ERR_INVALID_VARIANT;
        lc_variant vg = *v;
        const bool node = v->layout == LC_LAYOUT_NODE_MAJOR;
        for (int q = 0; q < 8 && G.E > 0 && rs != LC_OK; ++q) {
            vg = *v;
            if (q & 1)
                vg.stages = 1;
            if (q & 2)
                vg.elems_per_thread = v->elems_per_thread == 64 ? 1 : 64;
            if (q & 4) {
                if (node)
                    continue;
                vg.store_rows = 32;
            }
            if (q > 0 && memcmp(&vg, v, sizeof vg) == 0)
                continue;
            // three terms: the A terms in shared memory unless tensor memory is asked for; a
            // group whose three-term plan needs them in tensor memory runs as its own launch
            // after the grouped one (grouped_plan_all)
            if (T.nterms == 3 && v->a_operand == 0)
                vg.a_operand = 1;
            rs = resolve(K, G.E, G.N, G.F, &vg, r, true);
            if (rs == LC_ERR_NO_DEVICE || rs == LC_ERR_CUDA || rs == LC_ERR_INVALID_ARGUMENT ||
                rs == LC_ERR_ASSUMPTION)
                return rs;
        }
        if (rs != LC_OK) {
            T.simt_groups.push_back(gi);  // no tensor-core plan (or nothing to do)
            continue;
        }
        T.gv[gi] = vg;
        TcArgs t = r.tc;
        t.D = static_cast<const float *>(G.D_dev);
        t.u = static_cast<const float *>(G.u_dev);
        t.out = static_cast<float *>(G.out_dev);
        t.r = nullptr;
        t.err = error_word();
        t.chunk = 8;  // one kernel instance for all groups: 8-column epilogue chunks
        const int tg = (int)T.tc_groups.size();
        T.P.g[tg] = t;
        T.tc_groups.push_back(gi);
        T.smem = std::max(T.smem, (size_t)t.smem_bytes);
        T.threads = tc_threads(t);
        // per tile: its HBM bytes at the SM's share of the copy rate (0.6 efficiency), or the
        // MMA chain at about 300 cycles an instruction, plus a fixed pipeline cost
        const int kn = t.Kt;
        const int mmas = (T.nterms == 1 ? 1 : (t.stack ? 5 : 6)) * (kn / 16);
        for (int b = 0; b < t.nblocks; ++b) {
            const int gb = std::min(t.G, G.F - b * t.G);
            const double bytes = 128.0 * G.N * 4.0 * (1 + gb);
            const double cost = std::max(bytes / (6.7e12 / sms) / 0.6, mmas * 300.0 / 1.9e9) + 4e-7;
            units.push_back({tg, b, t.ntiles, cost});
        }
    }
    T.P.ngroups = (int)T.tc_groups.size();
    if (units.empty())
        return LC_OK;
    if ((int)units.size() > sms)
        return LC_ERR_INVALID_VARIANT;  // more units than SMs: one CTA per unit does not fit
    std::vector<int> n(units.size(), 1);
    int used = (int)units.size();
    while (used < sms) {
        size_t m = units.size();
        double worst = -1;
        for (size_t q = 0; q < units.size(); ++q) {
            if (n[q] >= units[q].tiles)
                continue;
            const double load = units[q].tiles * units[q].cost / n[q];
            if (load > worst) {
                worst = load;
                m = q;
            }
        }
        if (m == units.size())
            break;
        ++n[m];
        ++used;
    }
    for (size_t q = 0; q < units.size(); ++q)
        for (int r = 0; r < n[q]; ++r)
            T.map.push_back(make_int4(units[q].g, units[q].blk, r, n[q]));
    T.grid = (int)T.map.size();
    return LC_OK;
}

// The SIMT descriptor that serves the groups of a tensor-core grouped plan without a tensor
// plan (8 x 8 register blocks, unroll 4, two stages, three CTAs per SM: the fastest grouped
// SIMT shape measured on the uneven-batching workload).
static lc_variant grouped_simt_fallback(const lc_variant *v)
{
    lc_variant s;
    memset(&s, 0, sizeof s);
    s.struct_size = sizeof(lc_variant);
    s.engine = LC_ENGINE_SIMT;
    s.layout = v->layout;
    s.precision = LC_PREC_FP32;
    s.elems_per_thread = 8;
    s.split_i = 8;
    s.tile_e = 64;
    s.unroll = 4;
    s.prefetch_smem = 1;
    s.stages = 2;
    s.ctas_per_sm = 3;
    return s;
}

// Both parts of a grouped plan and the workspace layout: SIMT tables first, then the tensor
// part's unit table (16-byte aligned).
struct GroupedPlanAll {
    GroupedPlanHost S;
    GroupedPlanTc T;
    std::vector<lc_group> simt_groups;
    std::vector<int> simt_gi;  // their indices among the caller's groups
    lc_variant simt_v, ks_v, tcl_v;
    std::vector<KsLaunch> ks;
    std::vector<TcLaunch> tcl;
    bool has_simt = false;
    size_t off_map = 0, bytes = 0;
};

// The K-split descriptor for the groups of a grouped plan that run as their own K-split
// launch: tensor-core plans' groups without any tensor-core plan (N above 128 for three
// terms), FP32 plans' groups of N >= 96 (tiles of 128 elements, j chunks of 8, one u buffer:
// the fastest measured for N = 120 and 165).
static lc_variant grouped_ks_fallback(const lc_variant *v)
{
    lc_variant s;
    memset(&s, 0, sizeof s);
    s.struct_size = sizeof(lc_variant);
    s.engine = LC_ENGINE_KSPLIT;
    s.layout = v->layout;
    s.precision = LC_PREC_FP32;
    s.tile_e = 128;
    s.elems_per_thread = 8;
    s.split_i = 8;
    s.unroll = 8;
    s.prefetch_smem = 1;
    s.stages = 1;
    return s;
}

// The tensor-core descriptor for the groups of a three-term grouped plan without a shared-
// memory plan: the A terms where the planner puts them (tensor memory), one operator per
// column block, 32-row stores (the library's default there; N = 120: 0.44 ms against 0.69 ms
// for the K-split kernel).
static lc_variant grouped_tc_fallback(const lc_variant *v)
{
    lc_variant s;
    memset(&s, 0, sizeof s);
    s.struct_size = sizeof(lc_variant);
    s.engine = LC_ENGINE_TCGEN05;
    s.layout = v->layout;
    s.precision = v->precision;
    s.tile_e = 128;
    s.elems_per_thread = 64;
    s.split_i = 1;
    s.unroll = 3;
    s.prefetch_smem = 1;
    s.stages = 1;
    s.store_rows = v->layout == LC_LAYOUT_ELEM_MAJOR ? 32 : 0;
    return s;
}

// A K-split launch for group gi if its plan resolves (false: no K-split plan).
static lc_status grouped_add_ks(const Kernel &K, const lc_variant &kv, const lc_group &G, int gi,
                                std::vector<KsLaunch> &ks, bool *added)
{
    *added = false;
    Resolved r;
    const lc_status rs = resolve(K, G.E, G.N, G.F, &kv, r, true);
    if (rs == LC_ERR_NO_DEVICE || rs == LC_ERR_CUDA)
        return rs;
    if (rs != LC_OK)
        return LC_OK;
    KsLaunch L;
    L.a = r.ks;
    L.a.D = static_cast<const float *>(G.D_dev);
    L.a.u = static_cast<const float *>(G.u_dev);
    L.a.out = static_cast<float *>(G.out_dev);
    L.grid = r.g.grid;
    L.bm = r.ks_bm;
    L.bk = r.ks_bk;
    L.group = gi;
    ks.push_back(L);
    *added = true;
    return LC_OK;
}

static lc_status grouped_plan_all(const Kernel &K, const lc_variant *v, const lc_group *groups, int ng,
                                  GroupedPlanAll &A)
{
    if (!v || v->struct_size != sizeof(lc_variant) || !groups || ng <= 0)
        return LC_ERR_INVALID_ARGUMENT;
    if (v->engine != LC_ENGINE_TCGEN05) {
        // FP32: the groups of N >= 96 (where the K-split kernel, which streams D^T in chunks,
        // is the library's default) run as one K-split launch each after the persistent launch
        lc_status st = grouped_plan_host(K, v, groups, ng, A.S);  // validates the descriptor
        if (st != LC_OK)
            return st;
        if (v->precision == LC_PREC_FP32) {
            A.ks_v = grouped_ks_fallback(v);
            for (int gi = 0; gi < ng; ++gi) {
                const lc_group &G = groups[gi];
                bool added = false;
                if (G.E > 0 && G.N >= 96) {
                    st = grouped_add_ks(K, A.ks_v, G, gi, A.ks, &added);
                    if (st != LC_OK)
                        return st;
                }
                if (!added) {
                    A.simt_groups.push_back(G);
                    A.simt_gi.push_back(gi);
                }
            }
            if (!A.ks.empty()) {
                A.S = GroupedPlanHost();
                if (!A.simt_groups.empty()) {
                    st = grouped_plan_host(K, v, A.simt_groups.data(), (int)A.simt_groups.size(), A.S);
                    if (st != LC_OK)
                        return st;
                }
            }
        }
        A.has_simt = A.ks.empty() || !A.simt_groups.empty();
        A.bytes = A.has_simt ? A.S.bytes : 16;
        return LC_OK;
    }
    if (v->precision != LC_PREC_BF16 && v->precision != LC_PREC_BF16X3)
        return LC_ERR_INVALID_VARIANT;
    lc_status st = grouped_plan_tc(K, v, groups, ng, A.T);
    if (st != LC_OK)
        return st;
    // the rest: three terms, one tensor-core launch each with the A terms in tensor memory
    // where that plan resolves; else one K-split launch each; else (no K-split plan) the SIMT
    // grouped launch
    A.ks_v = grouped_ks_fallback(v);
    A.tcl_v = grouped_tc_fallback(v);
    for (int gi : A.T.simt_groups) {
        const lc_group &G = groups[gi];
        if (G.E == 0)
            continue;
        if (v->precision == LC_PREC_BF16X3) {
            Resolved r;
            const lc_status rs = resolve(K, G.E, G.N, G.F, &A.tcl_v, r, true);
            if (rs == LC_ERR_NO_DEVICE || rs == LC_ERR_CUDA)
                return rs;
            if (rs == LC_OK) {
                TcLaunch L;
                L.a = r.tc;
                L.a.D = static_cast<const float *>(G.D_dev);
                L.a.u = static_cast<const float *>(G.u_dev);
                L.a.out = static_cast<float *>(G.out_dev);
                L.a.err = error_word();
                L.layout = r.layout;
                L.nterms = 3;
                L.grid = r.tc_grid;
                L.group = gi;
                A.tcl.push_back(L);
                continue;
            }
        }
        bool added = false;
        const lc_status sk = grouped_add_ks(K, A.ks_v, G, gi, A.ks, &added);
        if (sk != LC_OK)
            return sk;
        if (!added) {
            A.simt_groups.push_back(G);
            A.simt_gi.push_back(gi);
        }
    }
    if (!A.simt_groups.empty()) {
        A.simt_v = grouped_simt_fallback(v);
        st = grouped_plan_host(K, &A.simt_v, A.simt_groups.data(), (int)A.simt_groups.size(), A.S);
        if (st != LC_OK)
            return st;
        A.has_simt = true;
    }
    A.off_map = A.has_simt ? (A.S.bytes + 15) / 16 * 16 : 0;
    A.bytes = A.off_map + sizeof(int4) * A.T.map.size();
    if (A.bytes == 0)
        A.bytes = 16;
    return LC_OK;
}

}  // namespace lc

lc_status lc_device_error(int clear)
{
    unsigned int *p = error_word();
    if (!p)
        return LC_ERR_NO_DEVICE;
    unsigned int h = 0;
    cudaError_t e = cudaMemcpy(&h, p, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (clear && h) {
        unsigned int z = 0;
        e = cudaMemcpy(p, &z, sizeof z, cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return cuda_fail(e);
    }
    return (h & 1u) ? LC_ERR_TIMEOUT : (h & 2u) ? LC_ERR_INDEX : LC_OK;
}

lc_status lc_grouped_workspace_size(const lc_kernel *kh, const lc_variant *v, const lc_group *groups,
                                    int32_t ngroups, size_t *bytes)
{
    if (!kh || !bytes)
        return LC_ERR_INVALID_ARGUMENT;
    GroupedPlanAll A;
    lc_status st = grouped_plan_all(kh->k, v, groups, ngroups, A);
    if (st != LC_OK)
        return st;
    *bytes = A.bytes;
    return LC_OK;
}

lc_status lc_grouped_plan_create(const lc_kernel *kh, const lc_variant *v, const lc_group *groups,
                                 int32_t ngroups, void *workspace, size_t workspace_bytes, int32_t use_graph,
                                 void *stream, lc_grouped_plan **out)
{
    if (!kh || !out || !workspace)
        return LC_ERR_INVALID_ARGUMENT;
    if (((uintptr_t)workspace & 15u) != 0)
        return LC_ERR_MISALIGNED;
    if (use_graph && !stream)
        return LC_ERR_INVALID_ARGUMENT;  // the legacy default stream cannot be captured
    int major = 0, minor = 0;
    if (current_cc(&major, &minor) != 0 || major != 10 || minor != 3)
        return LC_ERR_NO_DEVICE;
    GroupedPlanAll A;
    lc_status st = grouped_plan_all(kh->k, v, groups, ngroups, A);
    if (st != LC_OK)
        return st;
    if (workspace_bytes < A.bytes)
        return LC_ERR_BUFFER_TOO_SMALL;
    const GroupedPlanHost &P = A.S;
    const lc_variant *sv = v->engine == LC_ENGINE_TCGEN05 ? &A.simt_v : v;
    void *fn = nullptr;
    if (A.has_simt) {
        fn = grouped_kernel_ptr(sv->layout, sv->elems_per_thread, sv->split_i, sv->unroll, sv->prefetch_smem);
        if (!fn)
            return LC_ERR_INVALID_VARIANT;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    std::vector<unsigned char> host(A.bytes, 0);
    if (A.has_simt) {
        memcpy(host.data() + P.off_groups, P.groups.data(), sizeof(SimtArgs) * P.groups.size());
        memcpy(host.data() + P.off_segs, P.segs.data(), sizeof(GroupSeg) * P.segs.size());
        memcpy(host.data() + P.off_cta, P.cta_seg.data(), sizeof(int) * P.cta_seg.size());
    }
    if (!A.T.map.empty())
        memcpy(host.data() + A.off_map, A.T.map.data(), sizeof(int4) * A.T.map.size());
    cudaError_t e = cudaMemcpyAsync(ws, host.data(), A.bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && fn)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem);
    if (e != cudaSuccess)
        return cuda_fail(e);
    lc_grouped_plan *plan = new (std::nothrow) lc_grouped_plan;
    if (!plan)
        return LC_ERR_INVALID_ARGUMENT;
    if (A.has_simt) {
        plan->fn = fn;
        plan->args.groups = reinterpret_cast<const SimtArgs *>(ws + P.off_groups);
        plan->args.segs = reinterpret_cast<const GroupSeg *>(ws + P.off_segs);
        plan->args.cta_seg = reinterpret_cast<const int *>(ws + P.off_cta);
        plan->args.err = error_word();
        plan->grid = P.grid;
        plan->threads = P.threads;
        plan->smem = P.smem;
        plan->nsegs = (int)P.segs.size();
    }
    if (A.T.grid > 0) {
        plan->tcp = A.T.P;
        plan->tcp.map = reinterpret_cast<const int4 *>(ws + A.off_map);
        plan->grid_tc = A.T.grid;
        plan->threads_tc = A.T.threads;
        plan->smem_tc = A.T.smem;
        plan->nsegs += A.T.grid;
        st = tc_grouped_launch(plan->tcp, v->layout, A.T.nterms, 0, 0, plan->smem_tc, s, &plan->fn_tc);
        if (st != LC_OK) {
            delete plan;
            return st;
        }
    }
    plan->ngroups = ngroups;
    plan->group_variant.assign(ngroups, *v);
    if (v->engine == LC_ENGINE_TCGEN05) {
        for (int gi = 0; gi < ngroups; ++gi)
            plan->group_variant[gi] = A.T.gv[gi];
        for (int gi : A.simt_gi)
            plan->group_variant[gi] = A.simt_v;
    }
    for (const KsLaunch &L : A.ks)
        plan->group_variant[L.group] = A.ks_v;
    for (const TcLaunch &L : A.tcl)
        plan->group_variant[L.group] = A.tcl_v;
    plan->ks = A.ks;
    plan->tcl = A.tcl;
    plan->layout = v->layout;
    // shared-memory sizes, before any capture
    for (const KsLaunch &L : A.ks) {
        st = ks_launch(L.a, v->layout, L.bm, L.bk, 0, s, true);
        if (st != LC_OK) {
            delete plan;
            return st;
        }
    }
    for (const TcLaunch &L : A.tcl) {
        st = tc_launch(L.a, L.layout, L.nterms, 0, s);
        if (st != LC_OK) {
            delete plan;
            return st;
        }
    }
    if (use_graph) {
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = cudaSuccess;
            if (plan->fn_tc) {
                void *params[] = {&plan->tcp};
                le = cudaLaunchKernel(plan->fn_tc, dim3(plan->grid_tc), dim3(plan->threads_tc), params,
                                      plan->smem_tc, s);
            }
            for (const KsLaunch &L : plan->ks)
                if (le == cudaSuccess && ks_launch(L.a, plan->layout, L.bm, L.bk, L.grid, s, false) != LC_OK)
                    le = cudaErrorLaunchFailure;
            for (const TcLaunch &L : plan->tcl)
                if (le == cudaSuccess && tc_launch(L.a, L.layout, L.nterms, L.grid, s) != LC_OK)
                    le = cudaErrorLaunchFailure;
            if (le == cudaSuccess && plan->fn) {
                void *params[] = {&plan->args};
                le = cudaLaunchKernel(plan->fn, dim3(plan->grid), dim3(plan->threads), params, plan->smem, s);
            }
            e = cudaStreamEndCapture(s, &plan->graph);
            if (le != cudaSuccess)
                e = le;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        if (e != cudaSuccess) {
            if (plan->graph)
                cudaGraphDestroy(plan->graph);
            delete plan;
            return cuda_fail(e);
        }
    }
    *out = plan;
    return LC_OK;
}

lc_status lc_grouped_run(lc_grouped_plan *plan, void *stream)
{
    if (!plan)
        return LC_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (plan->exec) {
        e = cudaGraphLaunch(plan->exec, s);
    } else {
        if (plan->fn_tc) {
            void *params[] = {&plan->tcp};
            e = cudaLaunchKernel(plan->fn_tc, dim3(plan->grid_tc), dim3(plan->threads_tc), params, plan->smem_tc,
                                 s);
        }
        for (const KsLaunch &L : plan->ks) {
            if (e != cudaSuccess)
                break;
            const lc_status st = ks_launch(L.a, plan->layout, L.bm, L.bk, L.grid, s, false);
            if (st != LC_OK)
                return st;
        }
        for (const TcLaunch &L : plan->tcl) {
            if (e != cudaSuccess)
                break;
            const lc_status st = tc_launch(L.a, L.layout, L.nterms, L.grid, s);
            if (st != LC_OK)
                return st;
        }
        if (e == cudaSuccess && plan->fn) {
            void *params[] = {&plan->args};
            e = cudaLaunchKernel(plan->fn, dim3(plan->grid), dim3(plan->threads), params, plan->smem, s);
        }
    }
    if (e != cudaSuccess)
        return cuda_fail(e);
    return LC_OK;
}

lc_status lc_grouped_plan_info(const lc_grouped_plan *plan, int32_t *grid, int32_t *segments)
{
    if (!plan || !grid || !segments)
        return LC_ERR_INVALID_ARGUMENT;
    int g = plan->grid + plan->grid_tc;
    for (const KsLaunch &L : plan->ks)
        g += L.grid;
    for (const TcLaunch &L : plan->tcl)
        g += L.grid;
    *grid = g;
    *segments = plan->nsegs;
    return LC_OK;
}

lc_status lc_grouped_plan_group(const lc_grouped_plan *plan, int32_t group, lc_variant *v)
{
    if (!plan || !v || group < 0 || group >= plan->ngroups)
        return LC_ERR_INVALID_ARGUMENT;
    *v = plan->group_variant[group];
    return LC_OK;
}

void lc_grouped_plan_destroy(lc_grouped_plan *plan)
{
    if (!plan)
        return;
    if (plan->exec)
        cudaGraphExecDestroy(plan->exec);
    if (plan->graph)
        cudaGraphDestroy(plan->graph);
    delete plan;
}

lc_status lc_device_info(int32_t *sm, int32_t *major, int32_t *minor)
{
    if (!sm || !major || !minor)
        return LC_ERR_INVALID_ARGUMENT;
    int n = sm_count();
    if (n <= 0)
        return LC_ERR_NO_DEVICE;
    int a = 0, b = 0;
    if (current_cc(&a, &b) != 0)
        return LC_ERR_NO_DEVICE;
    *sm = n;
    *major = a;
    *minor = b;
    return LC_OK;
}

}  // extern "C"
