// planner.cpp -- host-side analysis of an HFAV rule DAG.
//
// Steps, in the order of the paper's method (Sec. 3, "Our transformation
// technique follows the following steps"):
//   1. dataflow DAG: validation (one producer per term, Sec. 2; acyclic,
//      Sec. 3.2) and a topological order of the callsites;
//   2./3. one perfect iteration nest per callsite group (Sec. 3.2.1-3.2.2);
//      reductions become init / accumulate / finalize phases placed in the
//      prologue / steady state / epilogue (Sec. 3.3.2);
//   4. fusion of the iteration-nest DAG in topological order with the
//      rank-ordering and dataflow-ordering rules (Sec. 3.3, Listings
//      "fuse_inest_dag" and "fuse_inest"); an unfusable pair is a split;
//   5. variable analysis: footprint by the Minkowski sum of offsets
//      (Sec. 3.5, footnote), enclosing region (which fields cross nests),
//      reuse order (Sec. 3.5 "Grouping"), contraction to rolling buffers
//      (Sec. 3.5 "Contraction");
//   6. instead of emitting C, the fusion groups are matched against the
//      hand-written GPU pipelines (recognise()).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <cctype>
#include <set>
#include <sstream>

#include "plan.hpp"

namespace hfav {

namespace {

bool op_known(int op) {
    switch (op) {
        case HFAV_OP_STENCIL_LINEAR: case HFAV_OP_GRADMAG_HALF: case HFAV_OP_SQUASH:
        case HFAV_OP_GENERIC: case HFAV_OP_LIMFLUX: case HFAV_OP_DIFFUSE: case HFAV_OP_EXPR: case HFAV_OP_CONSTOPRIM: case HFAV_OP_EOS: case HFAV_OP_SLOPE:
        case HFAV_OP_TRACE: case HFAV_OP_QLEFTRIGHT: case HFAV_OP_RIEMANN: case HFAV_OP_CMPFLX:
        case HFAV_OP_UPDATE: case HFAV_OP_CFL_DT: case HFAV_OP_REDUCE_SUM: case HFAV_OP_REDUCE_MAX: case HFAV_OP_BROADCAST:
            return true;
        default:
            return false;
    }
}

// the names a rule body may use besides in<k> / p<k>: the value type, casts
// and the CUDA math functions
bool allowed_name(const std::string& id) {
    static const std::set<std::string> names = {
        "T", "double", "float", "int", "sqrt", "rsqrt", "cbrt", "exp", "exp2", "expm1", "log", "log2",
        "log10", "log1p", "pow", "sin", "cos", "tan", "asin", "acos", "atan", "atan2", "sinh", "cosh",
        "tanh", "asinh", "acosh", "atanh", "fabs", "fmin", "fmax", "fma", "floor", "ceil", "trunc", "round",
        "rint", "copysign", "fmod", "hypot", "erf", "erfc", "tgamma", "lgamma", "fdim"};
    return names.count(id) != 0;
}

// A user rule body may only be an arithmetic expression: no statements,
// blocks, preprocessor lines, strings, comments, subscripts or addresses (no
// ';', '{', '#', quotes, '[', single '&'), and every name is one of the
// rule's inputs in<k> / parameters p<k> or an allowed type or math function
// -- so a body reads nothing but its inputs.
std::string check_expr(const char* e, int n_in, int n_params) {
    if (!e) return "an EXPR rule needs an expression";
    const size_t n = std::strlen(e);
    if (n == 0 || n > 4096) return "the expression must have 1 to 4096 characters";
    static const char ok[] = "_ .+-*<>/%()!=&|?:,^~";
    for (size_t k = 0; k < n; ++k) {
        const char c = e[k];
        if (!std::isalnum((unsigned char)c) && !std::strchr(ok, c) ) return std::string("character '") + c + "' is not allowed";
    }
    if (std::strstr(e, "/*") || std::strstr(e, "//")) return "comments are not allowed";
    for (size_t k = 0; k < n; ++k)   // no address-of (the only way to form a pointer)
        if (e[k] == '&') {
            if (k + 1 < n && e[k + 1] == '&') { ++k; continue; }
            return "'&' is only allowed as '&&'";
        }
    for (size_t k = 0; k < n;) {
        if (std::isalpha((unsigned char)e[k]) || e[k] == '_') {
            size_t b = k;
            while (k < n && (std::isalnum((unsigned char)e[k]) || e[k] == '_')) ++k;
            const std::string id(e + b, k - b);
            auto index_of = [&](const char* pre) -> long {
                const size_t m = std::strlen(pre);
                if (id.size() <= m || id.compare(0, m, pre) != 0) return -1;
                for (size_t q = m; q < id.size(); ++q)
                    if (!std::isdigit((unsigned char)id[q])) return -1;
                return id.size() - m > 6 ? 1000000 : std::stol(id.substr(m));
            };
            long a = index_of("in"), b2 = index_of("p");
            if (a >= n_in) return "'" + id + "' names an input the rule does not have";
            if (b2 >= n_params) return "'" + id + "' names a parameter the rule does not have";
            if (a < 0 && b2 < 0 && !allowed_name(id)) return "'" + id + "' is not an input, a parameter or a math function";
        } else if (std::isdigit((unsigned char)e[k]) || e[k] == '.') {
            while (k < n && (std::isalnum((unsigned char)e[k]) || e[k] == '.' ||
                             ((e[k] == '+' || e[k] == '-') && (e[k - 1] == 'e' || e[k - 1] == 'E'))))
                ++k;
        } else {
            ++k;
        }
    }
    return "";
}

// A rule is a reduction when it writes only rank-0 fields from higher-rank inputs.
bool is_reduction(const Dag& d, const Rule& r) {
    int in_rank = 0, out_rank = 0;
    for (auto& x : r.in) in_rank = std::max(in_rank, d.rank[x.field]);
    for (int f : r.out) out_rank = std::max(out_rank, d.rank[f]);
    return out_rank == 0 && in_rank > 0;
}

int rule_rank(const Dag& d, const Rule& r) {
    int rk = 0;
    for (int f : r.out) rk = std::max(rk, d.rank[f]);
    if (is_reduction(d, r))
        for (auto& x : r.in) rk = std::max(rk, d.rank[x.field]);
    return rk;
}

// Global loop order, outermost first: the stream axis, then the remaining
// axes from the highest index down (i, axis 0, innermost).
std::vector<int> loop_order(const Dag& d) {
    std::vector<int> o{d.stream_axis};
    for (int a = d.ndim - 1; a >= 0; --a)
        if (a != d.stream_axis) o.push_back(a);
    return o;
}

// ---- dataflow nodes: one per rule, three (init / acc / fin) per reduction --
struct Nodes {
    // node id = 3 * rule + part; part 0 = body or init, 1 = acc, 2 = fin
    int n = 0;
    std::vector<std::vector<uint64_t>> reach;   // reach[a] bit b: b depends (transitively) on a
    bool depends(int later, int earlier) const {
        return (reach[earlier][later >> 6] >> (later & 63)) & 1u;
    }
};

}  // namespace

std::string Schedule::str() const {
    static const char* fz[] = {"full", "sweep", "unfused"};
    static const char* pl[] = {"reg", "smem", "hbm"};
    char b[64];
    snprintf(b, sizeof b, "%s:%s:%dx%d", fz[fusion], pl[placement], tx, ty);
    return b;
}

bool parse_schedule(const char* s, Schedule* out, std::string* err) {
    Schedule r;
    if (!s || !*s || !strcmp(s, "auto")) { *out = r; return true; }
    std::string str(s);
    std::vector<std::string> parts;
    std::stringstream ss(str);
    std::string tok;
    while (std::getline(ss, tok, ':')) parts.push_back(tok);
    if (parts.empty() || parts.size() > 3) { *err = "schedule: expected fusion[:placement][:TXxTY]"; return false; }
    if (parts[0] == "full") r.fusion = FUSE_FULL;
    else if (parts[0] == "sweep") r.fusion = FUSE_SWEEP;
    else if (parts[0] == "unfused") { r.fusion = FUSE_UNFUSED; r.placement = PLACE_HBM; }
    else { *err = "schedule: unknown fusion '" + parts[0] + "'"; return false; }
    for (size_t k = 1; k < parts.size(); ++k) {
        const std::string& p = parts[k];
        if (p == "reg") r.placement = PLACE_REG;
        else if (p == "smem") r.placement = PLACE_SMEM;
        else if (p == "hbm") r.placement = PLACE_HBM;
        else {
            int tx = 0, ty = 0;
            if (sscanf(p.c_str(), "%dx%d", &tx, &ty) != 2 || tx <= 0 || ty <= 0) {
                *err = "schedule: bad component '" + p + "'"; return false;
            }
            r.tx = tx; r.ty = ty;
        }
    }
    if (r.fusion == FUSE_UNFUSED && r.placement != PLACE_HBM) {
        *err = "schedule: unfused implies hbm intermediates"; return false;
    }
    *out = r;
    return true;
}

int copy_dag(const hfav_dag* in, Dag* d) {
    if (!in) return set_error(HFAV_EINVAL, "dag is NULL");
    if (in->ndim < 1 || in->ndim > 3) return set_error(HFAV_EINVAL, "ndim must be 1, 2 or 3");
    if (in->stream_axis < 0 || in->stream_axis >= in->ndim)
        return set_error(HFAV_EINVAL, "stream_axis out of range");
    if (in->n_fields <= 0 || !in->field_rank) return set_error(HFAV_EINVAL, "no fields");
    if (in->n_rules <= 0 || !in->rules) return set_error(HFAV_EINVAL, "no rules");
    d->n_fields = in->n_fields;
    d->ndim = in->ndim;
    d->stream_axis = in->stream_axis;
    d->feedback = in->feedback;
    d->rank.assign(in->field_rank, in->field_rank + in->n_fields);
    for (int r : d->rank)
        if (r < 0 || r > in->ndim) return set_error(HFAV_EINVAL, "field rank out of range");
    auto fid_ok = [&](int f) { return f >= 0 && f < in->n_fields; };
    for (int i = 0; i < in->n_rules; ++i) {
        const hfav_rule& s = in->rules[i];
        Rule r;
        r.op = s.op; r.axis = s.axis;
        if (!op_known(s.op)) return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": unknown op");
        if (s.n_in < 0 || s.n_out < 1 || (s.n_in > 0 && !s.in) || !s.out || s.n_params < 0 ||
            (s.n_params > 0 && !s.params))
            return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": bad in/out/params");
        if (s.axis < 0 || s.axis >= in->ndim)
            return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": axis out of range");
        for (int k = 0; k < s.n_in; ++k) {
            if (!fid_ok(s.in[k].field)) return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": bad input field");
            for (int a = in->ndim; a < 3; ++a)
                if (s.in[k].off[a] != 0) return set_error(HFAV_EINVAL, "offset along an unused axis");
            r.in.push_back(s.in[k]);
        }
        for (int k = 0; k < s.n_out; ++k) {
            if (!fid_ok(s.out[k])) return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": bad output field");
            r.out.push_back(s.out[k]);
        }
        r.params.assign(s.params, s.params + s.n_params);
        if (s.op == HFAV_OP_EXPR) {
            const std::string why = check_expr(s.expr, s.n_in, s.n_params);
            if (!why.empty()) return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": " + why);
            if (s.n_out != 1) return set_error(HFAV_EINVAL, "rule " + std::to_string(i) + ": an EXPR rule has one output");
            r.expr = s.expr;
        }
        d->rules.push_back(r);
    }
    if (in->n_axioms < 0 || in->n_goals < 1 || (in->n_axioms > 0 && !in->axioms) || !in->goals)
        return set_error(HFAV_EINVAL, "bad axioms / goals");
    for (int k = 0; k < in->n_axioms; ++k) {
        if (!fid_ok(in->axioms[k])) return set_error(HFAV_EINVAL, "bad axiom field");
        d->axioms.push_back(in->axioms[k]);
    }
    for (int k = 0; k < in->n_goals; ++k) {
        if (!fid_ok(in->goals[k])) return set_error(HFAV_EINVAL, "bad goal field");
        d->goals.push_back(in->goals[k]);
    }
    if (d->feedback && d->axioms.size() != d->goals.size())
        return set_error(HFAV_EINVAL, "feedback needs as many goals as axioms");
    d->inout.assign(d->goals.size(), -1);
    if (in->inout) {
        if (d->feedback) return set_error(HFAV_EINVAL, "in/out aliasing cannot be declared with feedback");
        std::vector<char> used(d->axioms.size(), 0);
        for (size_t g = 0; g < d->goals.size(); ++g) {
            const int a = in->inout[g];
            if (a == -1) continue;
            if (a < 0 || a >= (int)d->axioms.size()) return set_error(HFAV_EINVAL, "inout: axiom index out of range");
            if (used[a]) return set_error(HFAV_EINVAL, "inout: an axiom aliased by two goals");
            if (d->rank[d->axioms[a]] != d->rank[d->goals[g]])
                return set_error(HFAV_EINVAL, "inout: aliased fields of different rank");
            used[a] = 1;
            d->inout[g] = a;
        }
    }
    return HFAV_OK;
}

// ---------------------------------------------------------------------------
// analysis
// ---------------------------------------------------------------------------
int analyze(hfav_plan_t* p, const int64_t* extent_in) {
    const Dag& d = p->dag;
    Analysis& A = p->an;
    const int nr = (int)d.rules.size(), nf = d.n_fields;
    int64_t extent[3] = {1, 1, 1};
    if (extent_in)
        for (int a = 0; a < d.ndim; ++a) extent[a] = extent_in[a];

    // --- 1. validation: producers, axioms, goals (Sec. 2, Sec. 3.2) -------
    std::vector<int> producer(nf, -1);
    std::vector<char> is_axiom(nf, 0), is_goal(nf, 0);
    for (int f : d.axioms) {
        if (is_axiom[f]) return set_error(HFAV_EINVAL, "axiom listed twice");
        is_axiom[f] = 1;
    }
    for (int f : d.goals) {
        if (is_goal[f]) return set_error(HFAV_EINVAL, "goal listed twice");
        is_goal[f] = 1;
    }
    for (int r = 0; r < nr; ++r)
        for (int f : d.rules[r].out) {
            if (is_axiom[f])
                return set_error(HFAV_EPRODUCER, "field " + std::to_string(f) + " is an axiom and is produced by rule " + std::to_string(r));
            if (producer[f] >= 0)
                return set_error(HFAV_EPRODUCER, "field " + std::to_string(f) + " has two producers (rules " +
                                                     std::to_string(producer[f]) + ", " + std::to_string(r) + ")");
            producer[f] = r;
        }
    for (int r = 0; r < nr; ++r)
        for (auto& x : d.rules[r].in)
            if (!is_axiom[x.field] && producer[x.field] < 0)
                return set_error(HFAV_EMISSING, "rule " + std::to_string(r) + " reads field " +
                                                    std::to_string(x.field) + ", which is neither an axiom nor produced");
    for (int f : d.goals)
        if (producer[f] < 0) return set_error(HFAV_EMISSING, "goal " + std::to_string(f) + " is never produced");

    // --- topological order (Kahn) -----------------------------------------
    std::vector<std::vector<int>> succ(nr);
    std::vector<int> indeg(nr, 0);
    for (int r = 0; r < nr; ++r) {
        std::set<int> preds;
        for (auto& x : d.rules[r].in)
            if (producer[x.field] >= 0) preds.insert(producer[x.field]);
        for (int q : preds) { succ[q].push_back(r); indeg[r]++; }
    }
    A.order.clear();
    {
        std::vector<int> ready;
        for (int r = 0; r < nr; ++r) if (!indeg[r]) ready.push_back(r);
        std::vector<int> deg = indeg;
        while (!ready.empty()) {
            std::sort(ready.begin(), ready.end(), std::greater<int>());
            int r = ready.back(); ready.pop_back();
            A.order.push_back(r);
            for (int s : succ[r]) if (--deg[s] == 0) ready.push_back(s);
        }
        if ((int)A.order.size() != nr) return set_error(HFAV_ECYCLE, "the rule graph has a cycle");
    }
    std::vector<int> topo_pos(nr);
    for (int k = 0; k < nr; ++k) topo_pos[A.order[k]] = k;

    // longest chain and largest offset (features for the cost model)
    {
        std::vector<int> depth(nr, 1);
        for (int r : A.order)
            for (int s : succ[r]) depth[s] = std::max(depth[s], depth[r] + 1);
        A.max_depth = nr ? *std::max_element(depth.begin(), depth.end()) : 0;
        A.max_radius = 0;
        for (auto& r : d.rules)
            for (auto& x : r.in)
                for (int a = 0; a < 3; ++a) A.max_radius = std::max(A.max_radius, std::abs(x.off[a]));
    }

    // --- dataflow nodes and reachability ----------------------------------
    Nodes N;
    N.n = 3 * nr;
    const int W64 = (N.n + 63) / 64;
    N.reach.assign(N.n, std::vector<uint64_t>(W64, 0));
    std::vector<char> red(nr, 0);
    for (int r = 0; r < nr; ++r) red[r] = is_reduction(d, d.rules[r]);
    auto out_node = [&](int r) { return red[r] ? 3 * r + 2 : 3 * r; };
    auto in_node = [&](int r) { return red[r] ? 3 * r + 1 : 3 * r; };
    std::vector<std::vector<int>> nsucc(N.n);
    for (int r = 0; r < nr; ++r) {
        if (red[r]) { nsucc[3 * r].push_back(3 * r + 1); nsucc[3 * r + 1].push_back(3 * r + 2); }
        std::set<int> preds;
        for (auto& x : d.rules[r].in)
            if (producer[x.field] >= 0) preds.insert(producer[x.field]);
        for (int q : preds) nsucc[out_node(q)].push_back(in_node(r));
    }
    // reverse topological sweep over rules (nodes inside a rule are ordered)
    for (int k = nr - 1; k >= 0; --k) {
        int r = A.order[k];
        int parts[3] = {3 * r + 2, 3 * r + 1, 3 * r};
        for (int pn : parts) {
            if (!red[r] && pn != 3 * r) continue;
            for (int s : nsucc[pn]) {
                N.reach[pn][s >> 6] |= 1ull << (s & 63);
                for (int w = 0; w < W64; ++w) N.reach[pn][w] |= N.reach[s][w];
            }
        }
    }

    // --- 2./3. initial iteration nests, one per rule ------------------------
    struct Nest {
        int irank;
        std::vector<int> prlg, steady, eplg;   // dataflow node ids
    };
    std::vector<Nest> nest(nr);
    for (int r = 0; r < nr; ++r) {
        Nest& n = nest[r];
        n.irank = rule_rank(d, d.rules[r]) - 1;   // rank of the outermost loop (-1: no loop)
        if (red[r]) { n.prlg = {3 * r}; n.steady = {3 * r + 1}; n.eplg = {3 * r + 2}; }
        else n.steady = {3 * r};
    }
    // dataflow_le(R, S): every node of R can be ordered before every node of S
    auto le = [&](const std::vector<int>& R, const std::vector<int>& S) {
        for (int a : R)
            for (int b : S)
                if (a == b || N.depends(a, b)) return false;   // a depends on b: b must precede a
        return true;
    };
    auto cat = [](std::vector<int> a, const std::vector<int>& b) { a.insert(a.end(), b.begin(), b.end()); return a; };
    // fuse_inest (Listing "fuse_inest"): same rank fuses phase-wise when the four
    // orderings hold; different ranks put the lower nest into the higher nest's
    // prologue (all of it can precede the steady state) or epilogue (the steady
    // state can precede all of it).  Returns false when unfusable (a split).
    auto fuse = [&](const Nest& A0, const Nest& B0, Nest* outn) -> bool {
        Nest A = A0, B = B0;
        if (A.irank == B.irank) {
            if (le(A.prlg, B.steady) && le(B.prlg, A.steady) && le(A.steady, B.eplg) && le(B.steady, A.eplg)) {
                outn->irank = A.irank;
                outn->prlg = cat(A.prlg, B.prlg);
                outn->steady = cat(A.steady, B.steady);
                outn->eplg = cat(A.eplg, B.eplg);
                return true;
            }
            return false;
        }
        if (A.irank > B.irank) std::swap(A, B);   // A is the lower-ranked nest
        std::vector<int> allA = cat(cat(A.prlg, A.steady), A.eplg);
        bool before = le(allA, B.steady) && le(allA, B.eplg);
        bool after = le(B.steady, allA) && le(B.prlg, allA);
        if (!before && !after) return false;
        outn->irank = B.irank;
        outn->steady = B.steady;
        if (before) { outn->prlg = cat(B.prlg, allA); outn->eplg = B.eplg; }
        else { outn->prlg = B.prlg; outn->eplg = cat(B.eplg, allA); }
        return true;
    };

    // --- 4. fuse_inest_dag: topological traversal with union of groups -----
    std::vector<int> grp(nr);
    for (int r = 0; r < nr; ++r) grp[r] = r;
    std::function<int(int)> find = [&](int x) { return grp[x] == x ? x : grp[x] = find(grp[x]); };
    std::map<int, Nest> gnest;
    for (int r = 0; r < nr; ++r) gnest[r] = nest[r];
    std::set<std::pair<int, int>> splits;   // rule pairs (producer, consumer) cut apart
    auto group_members = [&](int g) {
        std::vector<int> m;
        for (int r = 0; r < nr; ++r) if (find(r) == g) m.push_back(r);
        return m;
    };
    // merging groups a and b must not create a cycle through a third group
    auto creates_cycle = [&](int ga, int gb) {
        std::vector<int> ma = group_members(ga), mb = group_members(gb);
        auto rule_dep = [&](int later, int earlier) {   // rule later depends on rule earlier
            return N.depends(in_node(later), out_node(earlier)) || N.depends(3 * later + 0, out_node(earlier));
        };
        for (int x = 0; x < nr; ++x) {
            int gx = find(x);
            if (gx == ga || gx == gb) continue;
            bool from_a = false, to_b = false, from_b = false, to_a = false;
            for (int a : ma) { if (rule_dep(x, a)) from_a = true; if (rule_dep(a, x)) to_a = true; }
            for (int b : mb) { if (rule_dep(b, x)) to_b = true; if (rule_dep(x, b)) from_b = true; }
            if ((from_a && to_b) || (from_b && to_a)) return true;
        }
        return false;
    };
    for (int r : A.order) {
        std::set<int> preds;
        for (auto& x : d.rules[r].in)
            if (producer[x.field] >= 0) preds.insert(producer[x.field]);
        std::vector<int> pv(preds.begin(), preds.end());
        std::sort(pv.begin(), pv.end(), [&](int a, int b) { return topo_pos[a] > topo_pos[b]; });
        for (int q : pv) {
            int gv = find(r), gq = find(q);
            if (gv == gq) continue;
            Nest fused;
            if (fuse(gnest[gv], gnest[gq], &fused) && !creates_cycle(gv, gq)) {
                int keep = std::min(gv, gq), drop = std::max(gv, gq);
                grp[drop] = keep;
                gnest[keep] = fused;
                gnest.erase(drop);
            } else {
                splits.insert({q, r});
            }
        }
    }
    // group ids in topological order of first appearance
    std::map<int, int> gid;
    A.rule_group.assign(nr, -1);
    for (int r : A.order) {
        int g = find(r);
        if (!gid.count(g)) gid[g] = (int)gid.size();
        A.rule_group[r] = gid[g];
    }
    A.n_groups = (int)gid.size();
    A.group_rank.assign(A.n_groups, -1);
    for (auto& kv : gid) A.group_rank[kv.second] = gnest[kv.first].irank;

    // --- 5a. footprint: back-propagate the goal region (Minkowski sum) ------
    const int BIG = 1 << 28;
    std::vector<std::array<int, 3>> lo(nf), hi(nf);
    std::vector<char> set(nf, 0);
    for (int f = 0; f < nf; ++f) { lo[f] = {BIG, BIG, BIG}; hi[f] = {-BIG, -BIG, -BIG}; }
    for (int f : d.goals) { lo[f] = {0, 0, 0}; hi[f] = {0, 0, 0}; set[f] = 1; }
    for (int k = nr - 1; k >= 0; --k) {
        int r = A.order[k];
        const Rule& R = d.rules[r];
        std::array<int, 3> rlo = {BIG, BIG, BIG}, rhi = {-BIG, -BIG, -BIG};
        bool any = false;
        if (red[r]) { rlo = {0, 0, 0}; rhi = {0, 0, 0}; any = true; }   // reductions run over the interior
        else
            for (int f : R.out)
                if (set[f] && d.rank[f] > 0) {
                    any = true;
                    for (int a = 0; a < 3; ++a) { rlo[a] = std::min(rlo[a], lo[f][a]); rhi[a] = std::max(rhi[a], hi[f][a]); }
                }
        if (!any) { rlo = {0, 0, 0}; rhi = {0, 0, 0}; }
        // a rule runs over its outputs' footprint, which always holds the
        // interior (the reported halos are >= 0): its inputs must cover that
        // whole region, not only the part the consumers read
        for (int a = 0; a < d.ndim; ++a) { rlo[a] = std::min(rlo[a], 0); rhi[a] = std::max(rhi[a], 0); }
        for (auto& x : R.in) {
            if (d.rank[x.field] == 0) continue;
            set[x.field] = 1;
            for (int a = 0; a < d.ndim; ++a) {
                lo[x.field][a] = std::min(lo[x.field][a], rlo[a] + x.off[a]);
                hi[x.field][a] = std::max(hi[x.field][a], rhi[a] + x.off[a]);
            }
        }
    }

    // --- 5b. composed offsets per group (Sec. 3.5 Grouping / Contraction) ---
    // Within a fusion group, a field's references in one steady-state trip are
    // the offsets of its consumers composed back from the group's outputs.
    using Off = std::array<int, 3>;
    std::vector<std::set<Off>> offs(nf);      // composed offsets (max over groups by span)
    std::vector<std::array<int, 3>> win(nf), swin(nf);
    for (int f = 0; f < nf; ++f) { win[f] = {0, 0, 0}; swin[f] = {0, 0, 0}; }
    std::vector<std::vector<int>> consumers(nf);
    for (int r = 0; r < nr; ++r)
        for (auto& x : d.rules[r].in) consumers[x.field].push_back(r);
    for (int g = 0; g < A.n_groups; ++g) {
        std::vector<std::set<Off>> go(nf);
        std::vector<std::array<int, 3>> lead(nr, std::array<int, 3>{0, 0, 0});
        std::vector<char> has_lead(nr, 0);
        // seeds: outputs of the group that leave it (goals, other groups, scalars)
        for (int k = nr - 1; k >= 0; --k) {
            int r = A.order[k];
            if (A.rule_group[r] != g) continue;
            const Rule& R = d.rules[r];
            std::set<Off> ro;
            std::array<int, 3> ld = {-BIG, -BIG, -BIG};
            bool hl = false;
            for (int f : R.out) {
                bool leaves = is_goal[f] || d.rank[f] == 0;
                for (int c : consumers[f]) if (A.rule_group[c] != g) leaves = true;
                if (leaves) { go[f].insert(Off{0, 0, 0}); }
                for (auto& o : go[f]) ro.insert(o);
                // skewed lead: the furthest point any in-group consumer needs
                for (int c : consumers[f]) {
                    if (A.rule_group[c] != g || !has_lead[c]) continue;
                    for (auto& x : d.rules[c].in)
                        if (x.field == f)
                            for (int a = 0; a < 3; ++a) { ld[a] = std::max(ld[a], lead[c][a] + x.off[a]); hl = true; }
                }
            }
            if (ro.empty() || red[r]) ro.insert(Off{0, 0, 0});
            if (!hl || red[r]) ld = {0, 0, 0};
            lead[r] = ld; has_lead[r] = 1;
            for (auto& x : R.in) {
                if (d.rank[x.field] == 0) continue;
                for (auto& o : ro) go[x.field].insert(Off{o[0] + x.off[0], o[1] + x.off[1], o[2] + x.off[2]});
            }
        }
        for (int f = 0; f < nf; ++f) {
            if (go[f].empty()) continue;
            std::array<int, 3> w;
            for (int a = 0; a < 3; ++a) {
                int mn = BIG, mx = -BIG;
                for (auto& o : go[f]) { mn = std::min(mn, o[a]); mx = std::max(mx, o[a]); }
                w[a] = mx - mn + 1;
            }
            // skewed (software-pipelined) window: producer lead to the oldest in-group reference
            std::array<int, 3> sw = {1, 1, 1};
            bool any = false;
            std::array<int, 3> mn = {BIG, BIG, BIG}, mx = {-BIG, -BIG, -BIG};
            for (int c : consumers[f]) {
                if (A.rule_group[c] != g) continue;
                for (auto& x : d.rules[c].in)
                    if (x.field == f)
                        for (int a = 0; a < 3; ++a) {
                            any = true;
                            mn[a] = std::min(mn[a], lead[c][a] + x.off[a]);
                            mx[a] = std::max(mx[a], lead[c][a] + x.off[a]);
                        }
            }
            if (any) {
                int pr = producer[f];
                for (int a = 0; a < 3; ++a) {
                    int top = (pr >= 0 && A.rule_group[pr] == g) ? lead[pr][a] : mx[a];
                    sw[a] = std::max(top, mx[a]) - mn[a] + 1;
                }
            }
            int span_new = 1, span_old = 1;
            for (int a = 0; a < 3; ++a) { span_new *= w[a]; span_old *= std::max(1, win[f][a]); }
            if (offs[f].empty() || span_new > span_old) { offs[f] = go[f]; win[f] = w; }
            for (int a = 0; a < 3; ++a) swin[f][a] = std::max(swin[f][a], sw[a]);
        }
    }

    // --- 5c. per-field info: storage class, buffer size, reuse order --------
    std::vector<int> lord = loop_order(d);
    A.field.assign(nf, hfav_field_info{});
    for (int f = 0; f < nf; ++f) {
        hfav_field_info& fi = A.field[f];
        memset(&fi, 0, sizeof fi);
        fi.producer = producer[f];
        fi.group = producer[f] >= 0 ? A.rule_group[producer[f]] : -1;
        for (int a = 0; a < 3; ++a) {
            bool used = set[f] && a < d.ndim && d.rank[f] > 0;
            fi.halo_lo[a] = used ? std::max(0, -lo[f][a]) : 0;
            fi.halo_hi[a] = used ? std::max(0, hi[f][a]) : 0;
            fi.window[a] = std::max(1, win[f][a]);
            fi.stage_window[a] = std::max(1, swin[f][a]);
        }
        bool crosses = false;
        for (int c : consumers[f])
            if (producer[f] >= 0 && A.rule_group[c] != A.rule_group[producer[f]]) crosses = true;
        if (is_axiom[f]) fi.storage = HFAV_STORE_AXIOM;
        else if (is_goal[f]) fi.storage = HFAV_STORE_GOAL;
        else if (d.rank[f] == 0) fi.storage = HFAV_STORE_SCALAR;
        else if (crosses) fi.storage = HFAV_STORE_HBM;
        else fi.storage = HFAV_STORE_ROLLING;
        // rolling buffer: outer rotation (rows/planes) along the outermost axis
        // with span > 1, inner rotation (scalars) when only the innermost spans.
        int64_t elems = 1;
        for (size_t k = 0; k < lord.size(); ++k) {
            int a = lord[k];
            if (fi.window[a] > 1) {
                elems = fi.window[a];
                for (size_t m = k + 1; m < lord.size(); ++m) elems *= extent[lord[m]];
                break;
            }
        }
        if (fi.storage == HFAV_STORE_SCALAR) elems = 1;
        else if (fi.storage != HFAV_STORE_ROLLING) {
            elems = 1;
            for (int a = 0; a < d.ndim; ++a) elems *= extent[a] + fi.halo_lo[a] + fi.halo_hi[a];
        }
        fi.storage_elems = elems;
        // reuse order: the value at P is first touched by the trip whose offset
        // is largest in loop order, last by the smallest (a total order, so the
        // longest path of the "visited before" graph is this sorted list).
        std::vector<Off> ov(offs[f].begin(), offs[f].end());
        std::sort(ov.begin(), ov.end(), [&](const Off& x, const Off& y) {
            for (int a : lord) if (x[a] != y[a]) return x[a] > y[a];
            return false;
        });
        fi.n_reuse = (int)std::min<size_t>(ov.size(), 27);
        for (int k = 0; k < fi.n_reuse; ++k)
            for (int a = 0; a < 3; ++a) fi.reuse[k][a] = ov[k][a];
    }
    (void)splits;
    return HFAV_OK;
}

// ---------------------------------------------------------------------------
// pipeline recognition: map the DAG onto a hand-written fused kernel
// ---------------------------------------------------------------------------
namespace {

int box_index(const hfav_ref& x) {
    for (int a = 0; a < 3; ++a) if (x.off[a] < -1 || x.off[a] > 1) return -1;
    return (x.off[2] + 1) * 9 + (x.off[1] + 1) * 3 + (x.off[0] + 1);
}

bool take_linear(const Rule& r, int src, double* w) {
    if (r.op != HFAV_OP_STENCIL_LINEAR || r.in.size() != r.params.size() || r.out.size() != 1) return false;
    for (int k = 0; k < 27; ++k) w[k] = 0.0;
    std::set<int> seen;
    for (size_t k = 0; k < r.in.size(); ++k) {
        if (r.in[k].field != src) return false;
        int b = box_index(r.in[k]);
        if (b < 0 || seen.count(b)) return false;
        seen.insert(b);
        w[b] = r.params[k];
    }
    return true;
}

// gradient refs in the order (+1, -1) per axis, axes 0..n-1
bool take_grad(const Rule& r, int src, int naxes) {
    if (r.op != HFAV_OP_GRADMAG_HALF || (int)r.in.size() != 2 * naxes || r.out.size() != 1) return false;
    for (int a = 0; a < naxes; ++a)
        for (int s = 0; s < 2; ++s) {
            const hfav_ref& x = r.in[2 * a + s];
            if (x.field != src) return false;
            for (int b = 0; b < 3; ++b) {
                int want = (b == a) ? (s == 0 ? 1 : -1) : 0;
                if (x.off[b] != want) return false;
            }
        }
    return true;
}

bool take_squash(const Rule& r, int src) {
    return r.op == HFAV_OP_SQUASH && r.in.size() == 1 && r.in[0].field == src && r.out.size() == 1 &&
           r.in[0].off[0] == 0 && r.in[0].off[1] == 0 && r.in[0].off[2] == 0;
}

bool recognise_chain(hfav_plan_t* p) {
    const Dag& d = p->dag;
    const auto& o = p->an.order;
    if (d.axioms.size() != 1 || d.goals.size() != 1 || d.feedback) return false;
    int u = d.axioms[0];
    if (d.ndim == 2 && d.rules.size() == 3) {
        const Rule &a = d.rules[o[0]], &b = d.rules[o[1]], &c = d.rules[o[2]];
        for (int k = 0; k < 27; ++k) p->cmap.w1[k] = 0;
        if (!take_linear(a, u, p->cmap.w1)) return false;
        for (int k = 0; k < 27; ++k) if (k / 9 != 1 && p->cmap.w1[k] != 0.0) return false;
        if (!take_grad(b, a.out[0], 2) || !take_squash(c, b.out[0]) || c.out[0] != d.goals[0]) return false;
        if (d.stream_axis != 1) return false;
        p->cmap.rules[0] = o[0]; p->cmap.rules[1] = o[1]; p->cmap.rules[2] = o[2];
        p->pipeline = PIPE_CHAIN2D;
        return true;
    }
    if (d.ndim == 3 && d.rules.size() == 4) {
        const Rule &a = d.rules[o[0]], &b = d.rules[o[1]], &c = d.rules[o[2]], &e = d.rules[o[3]];
        if (!take_linear(a, u, p->cmap.w1) || !take_linear(b, a.out[0], p->cmap.w2)) return false;
        if (!take_grad(c, b.out[0], 3) || !take_squash(e, c.out[0]) || e.out[0] != d.goals[0]) return false;
        if (d.stream_axis != 2) return false;
        for (int k = 0; k < 4; ++k) p->cmap.rules[k] = o[k];
        p->pipeline = PIPE_CHAIN3D;
        return true;
    }
    return false;
}

// offset of one ref is exactly `want` (i, j, k)
bool off_is(const hfav_ref& x, int di, int dj, int dk) { return x.off[0] == di && x.off[1] == dj && x.off[2] == dk; }

// COSMO horizontal diffusion (Sec. 5.3): a 5-point star Laplacian of the
// axiom, LIMFLUX along i and along j of (u, lap), DIFFUSE into the goal, with
// the refs in the order the op catalogue states; 2D, or 3D with no k offsets.
bool recognise_cosmo(hfav_plan_t* p) {
    const Dag& d = p->dag;
    if (d.axioms.size() != 1 || d.goals.size() != 1 || d.feedback || d.rules.size() != 4) return false;
    if (d.ndim != 2 && d.ndim != 3) return false;
    const int u = d.axioms[0];
    const Rule* lap = nullptr;
    const Rule* fl[2] = {nullptr, nullptr};
    const Rule* up = nullptr;
    int lap_id = -1, fl_id[2] = {-1, -1}, up_id = -1;
    for (size_t k = 0; k < d.rules.size(); ++k) {
        const Rule& r = d.rules[k];
        if (r.op == HFAV_OP_STENCIL_LINEAR) { lap = &r; lap_id = (int)k; }
        else if (r.op == HFAV_OP_LIMFLUX && (r.axis == 0 || r.axis == 1)) { fl[r.axis] = &r; fl_id[r.axis] = (int)k; }
        else if (r.op == HFAV_OP_DIFFUSE) { up = &r; up_id = (int)k; }
    }
    if (!lap || !fl[0] || !fl[1] || !up) return false;
    double w[27];
    if (!take_linear(*lap, u, w)) return false;
    // a 5-point star in the (i, j) plane: box indices 13 centre, 14 / 12 i+-1, 16 / 10 j+-1
    for (int k = 0; k < 27; ++k)
        if (k != 13 && k != 14 && k != 12 && k != 16 && k != 10 && w[k] != 0.0) return false;
    const int L = lap->out[0];
    for (int a = 0; a < 2; ++a) {
        const Rule& r = *fl[a];
        const int di = a == 0, dj = a == 1;
        if (r.in.size() != 4 || r.out.size() != 1) return false;
        if (r.in[0].field != u || !off_is(r.in[0], 0, 0, 0) || r.in[1].field != u || !off_is(r.in[1], di, dj, 0) ||
            r.in[2].field != L || !off_is(r.in[2], 0, 0, 0) || r.in[3].field != L || !off_is(r.in[3], di, dj, 0))
            return false;
    }
    const int fx = fl[0]->out[0], fy = fl[1]->out[0];
    if (up->in.size() != 5 || up->out.size() != 1 || up->params.size() != 1 || up->out[0] != d.goals[0]) return false;
    if (up->in[0].field != u || !off_is(up->in[0], 0, 0, 0) || up->in[1].field != fx || !off_is(up->in[1], -1, 0, 0) ||
        up->in[2].field != fx || !off_is(up->in[2], 0, 0, 0) || up->in[3].field != fy ||
        !off_is(up->in[3], 0, -1, 0) || up->in[4].field != fy || !off_is(up->in[4], 0, 0, 0))
        return false;
    for (int k = 0; k < 27; ++k) p->cmap.w1[k] = w[k];
    p->cmap.coef = up->params[0];
    p->cmap.rules[0] = lap_id; p->cmap.rules[1] = fl_id[0]; p->cmap.rules[2] = fl_id[1]; p->cmap.rules[3] = up_id;
    p->pipeline = PIPE_COSMO;
    return true;
}

// Godunov: one rule of each Hydro2D op per axis (0 then 1), wired as the
// op catalogue in hfav.h states, plus an optional CFL_DT rule for dt.
bool recognise_godunov(hfav_plan_t* p) {
    const Dag& d = p->dag;
    if (d.ndim != 2 || d.axioms.size() != 4 || d.goals.size() != 4) return false;
    static const int ops[8] = {HFAV_OP_CONSTOPRIM, HFAV_OP_EOS, HFAV_OP_SLOPE, HFAV_OP_TRACE,
                               HFAV_OP_QLEFTRIGHT, HFAV_OP_RIEMANN, HFAV_OP_CMPFLX, HFAV_OP_UPDATE};
    int found[2][8];
    for (auto& a : found) for (int& x : a) x = -1;
    int cfl = -1;
    for (int r = 0; r < (int)d.rules.size(); ++r) {
        const Rule& R = d.rules[r];
        if (R.op == HFAV_OP_CFL_DT) { if (cfl >= 0) return false; cfl = r; continue; }
        int k = -1;
        for (int m = 0; m < 8; ++m) if (ops[m] == R.op) k = m;
        if (k < 0 || R.axis > 1 || found[R.axis][k] >= 0) return false;
        found[R.axis][k] = r;
    }
    for (auto& a : found) for (int x : a) if (x < 0) return false;
    if (cfl < 0) return false;
    const Rule& C = d.rules[cfl];
    if (C.in.size() != 4 || C.out.size() != 1 || d.rank[C.out[0]] != 0 || C.params.size() < 2) return false;
    for (int k = 0; k < 4; ++k)
        if (C.in[k].field != d.axioms[k]) return false;
    int dtf = C.out[0];
    double gamma = -1;
    // field wiring per axis
    std::vector<int> Uin(d.axioms.begin(), d.axioms.end());
    for (int ax = 0; ax < 2; ++ax) {
        const Rule* R[8];
        for (int k = 0; k < 8; ++k) R[k] = &d.rules[found[ax][k]];
        auto ref0 = [&](const hfav_ref& x, int f, int off) {
            for (int b = 0; b < 3; ++b) if (x.off[b] != (b == ax ? off : 0)) return false;
            return x.field == f;
        };
        // constoprim: U -> rho un ut e
        if (R[0]->in.size() != 4 || R[0]->out.size() != 4 || R[0]->params.size() < 1) return false;
        for (int k = 0; k < 4; ++k) if (!ref0(R[0]->in[k], Uin[k], 0)) return false;
        if (gamma < 0) gamma = R[0]->params[0];
        for (int k = 0; k < 8; ++k)
            if (R[k]->params.size() >= 1 && R[k]->params[0] != gamma) return false;
        if (R[5]->params.size() >= 2) {   // riemann: optional cap on the Newton iterations
            const double nm = R[5]->params[1];
            if (!(nm >= 1 && nm <= 10) || nm != (double)(int)nm) return false;
            if (ax == 1 && (int)nm != p->gmap.newton_max) return false;
            p->gmap.newton_max = (int)nm;
        } else if (ax == 1 && p->gmap.newton_max != 10) {
            return false;
        }
        const std::vector<int>& W = R[0]->out;   // rho un ut e
        // eos: rho e -> p c
        if (R[1]->in.size() != 2 || R[1]->out.size() != 2 || !ref0(R[1]->in[0], W[0], 0) || !ref0(R[1]->in[1], W[3], 0)) return false;
        int P = R[1]->out[0], Cc = R[1]->out[1];
        int prim[4] = {W[0], W[1], W[2], P};
        // slope: 12 refs q(-1) q(0) q(+1) for rho un ut p -> 4
        if (R[2]->in.size() != 12 || R[2]->out.size() != 4) return false;
        for (int q = 0; q < 4; ++q)
            for (int s = 0; s < 3; ++s)
                if (!ref0(R[2]->in[3 * q + s], prim[q], s - 1)) return false;
        // trace: rho un ut p c d[4] dt -> qm[4] qp[4]
        if (R[3]->in.size() != 10 || R[3]->out.size() != 8) return false;
        for (int q = 0; q < 4; ++q) if (!ref0(R[3]->in[q], prim[q], 0)) return false;
        if (!ref0(R[3]->in[4], Cc, 0)) return false;
        for (int q = 0; q < 4; ++q) if (!ref0(R[3]->in[5 + q], R[2]->out[q], 0)) return false;
        if (R[3]->in[9].field != dtf) return false;
        // qleftright: qp(0)[4] qm(+1)[4] -> qL qR
        if (R[4]->in.size() != 8 || R[4]->out.size() != 8) return false;
        for (int q = 0; q < 4; ++q) {
            if (!ref0(R[4]->in[q], R[3]->out[4 + q], 0)) return false;
            if (!ref0(R[4]->in[4 + q], R[3]->out[q], 1)) return false;
        }
        // riemann: qL qR -> g
        if (R[5]->in.size() != 8 || R[5]->out.size() != 4) return false;
        for (int q = 0; q < 8; ++q) if (!ref0(R[5]->in[q], R[4]->out[q], 0)) return false;
        // cmpflx: g -> F
        if (R[6]->in.size() != 4 || R[6]->out.size() != 4) return false;
        for (int q = 0; q < 4; ++q) if (!ref0(R[6]->in[q], R[5]->out[q], 0)) return false;
        // update: U F(0) F(-1) dt -> U'
        if (R[7]->in.size() != 13 || R[7]->out.size() != 4) return false;
        for (int q = 0; q < 4; ++q) {
            if (!ref0(R[7]->in[q], Uin[q], 0)) return false;
            if (!ref0(R[7]->in[4 + q], R[6]->out[q], 0)) return false;
            if (!ref0(R[7]->in[8 + q], R[6]->out[q], -1)) return false;
        }
        if (R[7]->in[12].field != dtf) return false;
        Uin = R[7]->out;
        for (int k = 0; k < 8; ++k) p->gmap.sweep_rules[ax][k] = found[ax][k];
    }
    for (int k = 0; k < 4; ++k) if (Uin[k] != d.goals[k]) return false;
    if (!d.feedback) return false;
    p->gmap.gamma = gamma;
    p->gmap.cfl = C.params[0];
    if (C.params[1] != gamma) return false;
    p->gmap.cfl_rule = cfl;
    p->pipeline = PIPE_GODUNOV;
    return true;
}

}  // namespace

int recognise(hfav_plan_t* p) {
    p->pipeline = PIPE_GENERIC;
    if (recognise_chain(p)) return HFAV_OK;
    if (recognise_godunov(p)) return HFAV_OK;
    if (recognise_cosmo(p)) return HFAV_OK;
    // generic DAGs of the stencil catalogue run unfused, one kernel per rule;
    // DAGs with user rule bodies or reductions get generated kernels.  Fields
    // are grid fields (rank ndim) or scalars (rank 0): a scalar comes from a
    // reduction of one grid field or from a rule body over scalars, and rule
    // bodies over the grid read scalars at offset 0 (broadcasts, Sec. 3.4)
    const Dag& d = p->dag;
    bool expr = false, scal = false;
    auto grid = [&](int f) { return d.rank[f] == d.ndim; };
    for (auto& r : d.rules) {
        if (r.out.size() != 1) return HFAV_EUNSUPPORTED;
        const int o = r.out[0];
        if (r.op == HFAV_OP_EXPR) {
            expr = true;
            bool reads_grid = false;
            for (auto& x : r.in) {
                if (grid(x.field) && !grid(o)) return HFAV_EUNSUPPORTED;   // grid -> scalar only by a reduction
                if (!grid(x.field) && (x.off[0] || x.off[1] || x.off[2])) return HFAV_EUNSUPPORTED;
                reads_grid = reads_grid || grid(x.field);
            }
            if (grid(o) && !reads_grid) return HFAV_EUNSUPPORTED;   // a grid field from scalars alone
            continue;
        }
        if (r.op == HFAV_OP_REDUCE_SUM || r.op == HFAV_OP_REDUCE_MAX) {
            if (r.in.size() != 1 || !grid(r.in[0].field) || d.rank[o] != 0) return HFAV_EUNSUPPORTED;
            scal = true;
            continue;
        }
        if (r.op != HFAV_OP_STENCIL_LINEAR && r.op != HFAV_OP_GRADMAG_HALF && r.op != HFAV_OP_SQUASH &&
            r.op != HFAV_OP_LIMFLUX && r.op != HFAV_OP_DIFFUSE)
            return HFAV_EUNSUPPORTED;
        for (auto& x : r.in) if (!grid(x.field)) return HFAV_EUNSUPPORTED;
        if (!grid(o)) return HFAV_EUNSUPPORTED;
    }
    for (int f = 0; f < d.n_fields; ++f) {
        if (grid(f)) continue;
        if (d.rank[f] != 0 || !scal) return expr ? HFAV_EUNSUPPORTED : HFAV_OK;
        for (int a : d.axioms) if (a == f) return HFAV_EUNSUPPORTED;
        for (int g : d.goals) if (g == f) return HFAV_EUNSUPPORTED;
    }
    if (scal && d.ndim != 2) return HFAV_EUNSUPPORTED;
    if (expr || scal) p->pipeline = PIPE_CODEGEN;
    return HFAV_OK;
}

bool schedule_valid(const hfav_plan_t* p, const Schedule& s, std::string* why) {
    static const int tiles[4][2] = {{32, 4}, {64, 4}, {128, 2}, {32, 8}};
    bool tile_ok = false;
    for (auto& t : tiles) if (t[0] == s.tx && t[1] == s.ty) tile_ok = true;
    if (!tile_ok) { if (why) *why = "tile must be one of 32x4, 64x4, 128x2, 32x8"; return false; }
    if (p->pipeline == PIPE_GENERIC && s.fusion != FUSE_UNFUSED) {
        if (why) *why = "this DAG has no fused GPU pipeline; use 'unfused'";
        return false;
    }
    if (s.fusion == FUSE_UNFUSED && s.placement != PLACE_HBM) {
        if (why) *why = "unfused implies hbm intermediates";
        return false;
    }
    if (p->pipeline == PIPE_CODEGEN && s.fusion != FUSE_UNFUSED) {
        if (s.fusion != FUSE_FULL || s.placement == PLACE_HBM || p->dag.ndim != 2) {
            if (why)
                *why = "generated kernels run fully fused on 2D DAGs -- shared-memory rings (full:smem) or warp strips "
                       "(full:reg) -- or unfused";
            return false;
        }
        if (s.placement == PLACE_REG && !codegen_wstrip_ok(p, s, why)) return false;
    }
    if (p->pipeline == PIPE_COSMO && s.fusion != FUSE_UNFUSED && (s.fusion != FUSE_FULL || s.placement != PLACE_REG)) {
        if (why) *why = "the COSMO pipeline runs fully fused with register windows (full:reg) or unfused";
        return false;
    }
    return true;
}

std::vector<Schedule> valid_schedules(const hfav_plan_t* p) {
    static const int tiles[4][2] = {{32, 4}, {64, 4}, {128, 2}, {32, 8}};
    std::vector<Schedule> v;
    for (int f = 0; f < 3; ++f)
        for (int pl = 0; pl < 3; ++pl)
            for (auto& t : tiles) {
                Schedule s;
                s.fusion = f; s.placement = pl; s.tx = t[0]; s.ty = t[1];
                if (schedule_valid(p, s, nullptr)) v.push_back(s);
            }
    return v;
}

std::string dump_json(const hfav_plan_t* p) {
    static const char* sto[] = {"axiom", "goal", "hbm", "rolling", "scalar"};
    static const char* pipes[] = {"generic", "chain2d", "chain3d", "godunov", "cosmo", "codegen"};
    const Analysis& A = p->an;
    std::ostringstream o;
    o << "{\"pipeline\":\"" << pipes[p->pipeline] << "\",\"schedule\":\"" << p->sched.str()
      << "\",\"n_groups\":" << A.n_groups << ",\"order\":[";
    for (size_t k = 0; k < A.order.size(); ++k) o << (k ? "," : "") << A.order[k];
    o << "],\"rule_group\":[";
    for (size_t k = 0; k < A.rule_group.size(); ++k) o << (k ? "," : "") << A.rule_group[k];
    o << "],\"fields\":[";
    for (size_t f = 0; f < A.field.size(); ++f) {
        const hfav_field_info& fi = A.field[f];
        o << (f ? "," : "") << "{\"id\":" << f << ",\"storage\":\"" << sto[fi.storage] << "\",\"group\":" << fi.group
          << ",\"halo_lo\":[" << fi.halo_lo[0] << "," << fi.halo_lo[1] << "," << fi.halo_lo[2] << "],\"halo_hi\":["
          << fi.halo_hi[0] << "," << fi.halo_hi[1] << "," << fi.halo_hi[2] << "],\"window\":[" << fi.window[0] << ","
          << fi.window[1] << "," << fi.window[2] << "],\"stage_window\":[" << fi.stage_window[0] << ","
          << fi.stage_window[1] << "," << fi.stage_window[2] << "],\"storage_elems\":" << fi.storage_elems << "}";
    }
    o << "]}";
    return o.str();
}

// Features for the learned schedule model.  They are the terms of a simple
// cost model of the schedule -- logs of the times its compulsory HBM bytes,
// its FP64 and FP32 operations (with the tile's halo recompute) and its
// on-chip staging would take at this GPU's measured rates, its launch count
// -- plus one-hot fusion / placement and the tile shape.  Expressed in time,
// they carry over between DAG families and dimensions (a 2D training set and
// a 3D held-out chain) better than raw sizes do.
void features(const hfav_plan_t* p, const Schedule& s, float* f) {
    for (int k = 0; k < HFAV_N_FEATURES; ++k) f[k] = 0.f;
    const Dag& d = p->dag;
    double cells = 0;
    for (auto& g : p->grids) cells += (double)g.extent[0] * g.extent[1] * g.extent[2];
    if (cells <= 0) cells = 1;
    const bool f64 = p->dtype == HFAV_F64;
    const double es = f64 ? 8.0 : 4.0;
    int n_inter = 0;
    for (auto& fi : p->an.field)
        if (fi.storage == HFAV_STORE_ROLLING || fi.storage == HFAV_STORE_HBM) n_inter++;
    const double R = p->an.max_radius;
    const int depth = p->an.max_depth;
    const int tiled = d.ndim - 1;   // axes the CTA tile covers (the stream axis is not tiled)
    // per cell and time step: FP64 / FP32 operations (times the recompute of
    // the kernel's halo), compulsory HBM bytes, on-chip operations (shared
    // memory, shuffles; global-memory staging and L1 loads count double) and
    // index arithmetic, as the kernel each schedule launches spends them
    double ops64 = 0, ops32 = 0, bytes = 0, chip = 0, iops = 0, launches = 1, rec = 1.0;
    const double TX = s.tx, TY = s.ty;
    const double gw = 2.0;   // weight of a global-memory (L1 / L2) operation
    if (p->pipeline == PIPE_GODUNOV) {
        const double it = 2.06, sweep = 155.0 + 40.0 * it;
        if (f64) ops64 = 2 * sweep + 16;
        else { ops64 = 2 * 36.0 * it; ops32 = 2 * sweep + 16 - ops64; }
        const double ywin = s.placement == PLACE_REG ? 0.0 : s.placement == PLACE_SMEM ? 60.0 : 60.0 * gw;
        const double xst = s.placement == PLACE_REG ? 40.0 : s.placement == PLACE_SMEM ? 40.0 : 40.0 * gw;
        if (s.fusion == FUSE_FULL) {
            bytes = 8 * es; chip = 40.0 + 8.0 + ywin; iops = 60; launches = 1;
            rec = TX / (TX - 2) * 1.15;
        } else if (s.fusion == FUSE_SWEEP) {
            bytes = 16 * es; chip = xst + ywin; iops = 60; launches = 2; rec = 1.03;
        } else {
            bytes = 74 * es; chip = 80.0 * gw; iops = 80 * 6; launches = 19;
        }
    } else {
        const bool c3 = p->pipeline == PIPE_CHAIN3D;
        const double ops = c3 ? 26.0 : p->pipeline == PIPE_CHAIN2D ? 14.0 : 8.0 * d.rules.size();
        const double io = (double)(d.axioms.size() + d.goals.size()) * es;
        double refs = 0, ax_refs = 0;
        for (auto& r : d.rules) {
            refs += r.in.size();
            for (auto& x : r.in)
                for (int f : d.axioms) if (x.field == f) ax_refs += 1;
        }
        double o32 = ops;
        if (s.fusion == FUSE_FULL) {
            bytes = io; iops = 2 * refs; launches = 1;
            if (c3) {
                // tile of outputs: TX x 16 (register windows; TX x 8 when TY = 2) or TX x TY (rings)
                const double oy = s.placement == PLACE_REG ? (TY >= 4 ? 16.0 : 8.0) : TY;
                const double ru = (TX + 6) * (oy + 6) / (TX * oy), r1 = (TX + 4) * (oy + 4) / (TX * oy),
                             r2 = (TX + 2) * (oy + 2) / (TX * oy);
                const double wr = ru + r1 + r2;
                chip = s.placement == PLACE_REG ? wr + 5 * r1 + 5 * r2 + 5 : (wr + 7 * r1 + 7 * r2 + 6);
                if (s.placement == PLACE_HBM) chip *= gw;
                o32 = 7 * r1 + 7 * r2 + 12;
            } else {
                const double rr = (TX + 2) / TX * 1.06;
                chip = s.placement == PLACE_REG ? 6.0 * 1.06 : 11.0 * rr;
                if (s.placement == PLACE_HBM) chip *= gw;
                o32 = ops * rr;
            }
        } else if (s.fusion == FUSE_SWEEP) {
            // first stage materialised by the generic kernel; the tail of the
            // 3D chain recomputes s2 at each gradient tap from s1
            bytes = io + 2 * es; launches = 2;
            const double first = d.rules.empty() ? 0 : d.rules[p->an.order[0]].in.size();
            const double tail = c3 ? 6.0 * 7.0 + 6.0 : 4.0;
            chip = (first + 1 + tail + 1) * gw;
            iops = first * (3 * 25.0) + tail * 6.0;
            o32 = c3 ? 7.0 + 6.0 * 7.0 + 12.0 : ops;
        } else {
            bytes = io + 2 * es * n_inter; launches = (double)d.rules.size();
            chip = (refs + d.rules.size()) * gw;
            iops = ax_refs * (3 * 25.0) + (refs - ax_refs) * 8.0;
        }
        (f64 ? ops64 : ops32) = o32;
    }
    const double us = 1e6;
    const double t_hbm = bytes * cells / 6.8e12 * us;
    const double t64 = ops64 * rec * cells / 5.9e11 * us;
    const double t32 = ops32 * cells / 6.9e13 * us;
    const double t_chip = chip * es * cells / 3.0e13 * us;
    const double t_int = iops * cells / 1.8e13 * us;
    const double t_launch = 3.0 * launches;
    // the analytic estimate the network corrects (microseconds per step)
    const double t_model = std::max(std::max(t_hbm, t_chip), std::max(t64, t32)) + t_int + t_launch;
    // scale-free inputs: how the estimate splits over resources, fusion,
    // placement, threads per CTA; the tile shape enters only through rec
    // (the same shape has one tiled axis in 2D and two in 3D)
    f[0] = (float)(std::log2(cells) / 24.0);
    f[1] = (float)(t_hbm / t_model);
    f[2] = (float)(t64 / t_model);
    f[3] = (float)(t32 / t_model);
    f[4] = (float)(t_chip / t_model);
    f[5] = (float)(t_int / t_model);
    f[6] = s.fusion == FUSE_FULL ? 1.f : 0.f;
    f[7] = s.fusion == FUSE_SWEEP ? 1.f : 0.f;
    f[8] = s.placement == PLACE_REG ? 1.f : 0.f;
    f[9] = s.placement == PLACE_SMEM ? 1.f : 0.f;
    f[10] = (float)(t_launch / t_model);
    f[11] = (float)(std::log2((double)s.tx * s.ty) / 8.0);
    f[HFAV_FEATURE_BASE] = (float)(std::log2(t_model) / 16.0);
    f[13] = s.fusion == FUSE_UNFUSED ? 1.f : 0.f;
    // resident warps per SM of the schedule's main kernel (register and
    // shared-memory limits of the compiled kernel); 24 when no device answers
    double warps = p->pipeline == PIPE_GODUNOV ? godunov_kernel_warps(p, s)
                   : (p->pipeline == PIPE_CHAIN2D || p->pipeline == PIPE_CHAIN3D) ? chain_kernel_warps(p, s) : -1.0;
    if (warps <= 0) warps = 24.0;
    f[14] = (float)(warps / 64.0);
    f[15] = f64 ? 1.f : 0.f;
}

}  // namespace hfav
