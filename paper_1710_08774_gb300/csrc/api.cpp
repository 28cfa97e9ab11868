// api.cpp -- extern "C" entry points declared in include/hfav.h.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "plan.hpp"

namespace hfav {
namespace {
thread_local std::string g_err;
}
int set_error(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
}  // namespace hfav

using namespace hfav;

namespace {

int copy_out(const std::string& s, char* buf, size_t n) {
    if (!buf || n == 0) return set_error(HFAV_EINVAL, "null buffer");
    size_t k = s.size() < n - 1 ? s.size() : n - 1;
    memcpy(buf, s.data(), k);
    buf[k] = 0;
    if (k < s.size()) return set_error(HFAV_EINVAL, "buffer too small: need " + std::to_string(s.size() + 1));
    return HFAV_OK;
}

int check_grids(hfav_plan_t* p) {
    const Dag& d = p->dag;
    for (size_t g = 0; g < p->grids.size(); ++g) {
        const hfav_grid& G = p->grids[g];
        if (G.pitch[0] != 1) return set_error(HFAV_EINVAL, "pitch[0] must be 1");
        for (int a = 0; a < 3; ++a)
            if (G.extent[a] < 1 || (a >= d.ndim && G.extent[a] != 1))
                return set_error(HFAV_EINVAL, "bad extent on axis " + std::to_string(a));
        if (G.halo < 0) return set_error(HFAV_EINVAL, "negative halo");
        // every axiom / goal array must hold the halo the analysis inferred
        int need = 0;
        for (int f : d.axioms)
            for (int a = 0; a < d.ndim; ++a) {
                need = std::max(need, p->an.field[f].halo_lo[a]);
                need = std::max(need, p->an.field[f].halo_hi[a]);
            }
        if (p->bc == HFAV_BC_HALO_GIVEN && G.halo < need)
            return set_error(HFAV_EHALO, "grid " + std::to_string(g) + ": halo " + std::to_string(G.halo) +
                                             " < inferred footprint " + std::to_string(need));
        int64_t row = G.extent[0] + 2 * G.halo;
        if (d.ndim >= 2 && G.pitch[1] < row) return set_error(HFAV_EHALO, "pitch[1] smaller than the padded row");
        if (d.ndim >= 3 && G.pitch[2] < G.pitch[1] * (G.extent[1] + 2 * G.halo))
            return set_error(HFAV_EHALO, "pitch[2] smaller than the padded plane");
        if (p->bc == HFAV_BC_PERIODIC)
            for (int a = 0; a < d.ndim; ++a) {
                int r = 0;
                for (size_t f = 0; f < p->an.field.size(); ++f)
                    r = std::max(r, std::max(p->an.field[f].halo_lo[a], p->an.field[f].halo_hi[a]));
                if (G.extent[a] < r)
                    return set_error(HFAV_EHALO, "periodic extent smaller than the stencil footprint");
            }
    }
    return HFAV_OK;
}

}  // namespace

extern "C" {

int hfav_version(void) { return 10100; }

const char* hfav_last_error(void) { return g_err.c_str(); }

int hfav_analyze(const hfav_dag* dag, const int64_t* extent, hfav_plan_t** out) {
    if (!out) return set_error(HFAV_EINVAL, "out is NULL");
    *out = nullptr;
    hfav_plan_t* p = new (std::nothrow) hfav_plan_s();
    if (!p) return set_error(HFAV_ENOMEM, "host allocation failed");
    p->analysis_only = true;
    int rc = copy_dag(dag, &p->dag);
    if (rc == HFAV_OK) rc = analyze(p, extent);
    if (rc == HFAV_OK) recognise(p);   // pipeline is informative only here
    if (rc != HFAV_OK) { delete p; return rc; }
    *out = p;
    return HFAV_OK;
}

int hfav_plan(const hfav_dag* dag, const hfav_grid* grids, int n_grids, int dtype, int bc,
              const char* schedule, hfav_plan_t** out) {
    if (!out) return set_error(HFAV_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grids || n_grids < 1) return set_error(HFAV_EINVAL, "need at least one grid");
    if (dtype != HFAV_F64 && dtype != HFAV_F32) return set_error(HFAV_EINVAL, "bad dtype");
    if (bc != HFAV_BC_PERIODIC && bc != HFAV_BC_HALO_GIVEN) return set_error(HFAV_EINVAL, "bad bc");
    hfav_plan_t* p = new (std::nothrow) hfav_plan_s();
    if (!p) return set_error(HFAV_ENOMEM, "host allocation failed");
    p->dtype = dtype;
    p->bc = bc;
    p->grids.assign(grids, grids + n_grids);
    int rc = copy_dag(dag, &p->dag);
    if (rc == HFAV_OK) rc = analyze(p, grids[0].extent);
    if (rc == HFAV_OK) rc = recognise(p);
    if (rc == HFAV_EUNSUPPORTED) set_error(rc, "no GPU kernels for some op of this DAG");
    if (rc == HFAV_OK) rc = check_grids(p);
    if (rc == HFAV_OK && p->pipeline == PIPE_GODUNOV && bc != HFAV_BC_PERIODIC)
        rc = set_error(HFAV_EUNSUPPORTED, "the Godunov pipeline runs on periodic grids only");
    if (rc == HFAV_OK && p->pipeline != PIPE_GODUNOV && n_grids != 1)
        rc = set_error(HFAV_EUNSUPPORTED, "batches of grids are supported for the Godunov pipeline only");
    // HFAV_SCHEDULE overrides a NULL / "auto" schedule argument: "auto", an
    // explicit variant, or "tuned" (autotune on the arrays of the first run)
    const char* env = getenv("HFAV_SCHEDULE");
    if (rc == HFAV_OK && (!schedule || !strcmp(schedule, "auto")) && env && *env) {
        if (!strcmp(env, "tuned")) p->tune_first_run = true;
        else schedule = env;
    }
    if (rc == HFAV_OK && schedule && !strcmp(schedule, "tuned")) { p->tune_first_run = true; schedule = nullptr; }
    if (rc == HFAV_OK) {
        Schedule s;
        std::string err;
        if (!parse_schedule(schedule, &s, &err)) rc = set_error(HFAV_EINVAL, err);
        else if (p->pipeline == PIPE_GENERIC && (!schedule || !strcmp(schedule, "auto"))) {
            s.fusion = FUSE_UNFUSED; s.placement = PLACE_HBM;
        } else if (p->pipeline == PIPE_CODEGEN && (!schedule || !strcmp(schedule, "auto"))) {
            // generated kernels: the fused shared-memory tile in 2D, else one kernel per rule
            if (p->dag.ndim == 2) { s.fusion = FUSE_FULL; s.placement = PLACE_SMEM; s.tx = 32; s.ty = 8; }
            else { s.fusion = FUSE_UNFUSED; s.placement = PLACE_HBM; }
        }
        if (rc == HFAV_OK && !schedule_valid(p, s, &err)) rc = set_error(HFAV_EUNSUPPORTED, err);
        if (rc == HFAV_OK) p->sched = s;
    }
    if (rc != HFAV_OK) { delete p; return rc; }
    *out = p;
    return HFAV_OK;
}

int hfav_plan_groups(const hfav_plan_t* p, int* n_groups, int* rule_group, int n_rules) {
    if (!p || !n_groups) return set_error(HFAV_EINVAL, "null argument");
    *n_groups = p->an.n_groups;
    if (rule_group) {
        if (n_rules < (int)p->dag.rules.size()) return set_error(HFAV_EINVAL, "rule_group too short");
        for (size_t r = 0; r < p->dag.rules.size(); ++r) rule_group[r] = p->an.rule_group[r];
    }
    return HFAV_OK;
}

int hfav_plan_order(const hfav_plan_t* p, int* order, int n_rules) {
    if (!p || !order || n_rules < (int)p->an.order.size()) return set_error(HFAV_EINVAL, "bad argument");
    for (size_t k = 0; k < p->an.order.size(); ++k) order[k] = p->an.order[k];
    return HFAV_OK;
}

int hfav_plan_field(const hfav_plan_t* p, int field, hfav_field_info* info) {
    if (!p || !info) return set_error(HFAV_EINVAL, "null argument");
    if (field < 0 || field >= (int)p->an.field.size()) return set_error(HFAV_EINVAL, "field out of range");
    *info = p->an.field[field];
    return HFAV_OK;
}

int hfav_plan_set_schedule(hfav_plan_t* p, const char* schedule) {
    if (!p || p->analysis_only) return set_error(HFAV_EINVAL, "not an executable plan");
    Schedule s;
    std::string err;
    if (!parse_schedule(schedule, &s, &err)) return set_error(HFAV_EINVAL, err);
    if (!schedule_valid(p, s, &err)) return set_error(HFAV_EUNSUPPORTED, err);
    p->sched = s;
    drop_graph(p);
    return HFAV_OK;
}

int hfav_plan_schedule(const hfav_plan_t* p, char* buf, size_t n) {
    if (!p) return set_error(HFAV_EINVAL, "null plan");
    return copy_out(p->sched.str(), buf, n);
}

int hfav_plan_dump(const hfav_plan_t* p, char* buf, size_t n) {
    if (!p) return set_error(HFAV_EINVAL, "null plan");
    return copy_out(dump_json(p), buf, n);
}

int hfav_plan_source(const hfav_plan_t* p, char* buf, size_t n) {
    if (!p || p->analysis_only) return set_error(HFAV_EINVAL, "not an executable plan");
    std::string src;
    int rc = plan_source(p, &src);
    return rc ? rc : copy_out(src, buf, n);
}

int hfav_plan_variants(const hfav_plan_t* p, char* buf, size_t n) {
    if (!p) return set_error(HFAV_EINVAL, "null plan");
    std::string s;
    auto v = valid_schedules(p);
    for (auto& x : v) s += x.str() + "\n";
    int rc = copy_out(s, buf, n);
    return rc == HFAV_OK ? (int)v.size() : rc;
}

int hfav_plan_features(const hfav_plan_t* p, const char* schedule, float* feat) {
    if (!p || !feat) return set_error(HFAV_EINVAL, "null argument");
    Schedule s = p->sched;
    std::string err;
    if (schedule && !parse_schedule(schedule, &s, &err)) return set_error(HFAV_EINVAL, err);
    features(p, s, feat);
    return HFAV_OK;
}

int hfav_run(hfav_plan_t* p, void* const* ax, void* const* go, int n_steps, void* stream) {
    if (!p || p->analysis_only) return set_error(HFAV_EINVAL, "not an executable plan");
    return run(p, ax, go, n_steps, stream, false);
}

int hfav_run_graph(hfav_plan_t* p, void* const* ax, void* const* go, int n_steps, void* stream) {
    if (!p || p->analysis_only) return set_error(HFAV_EINVAL, "not an executable plan");
    return run(p, ax, go, n_steps, stream, true);
}

int hfav_status(hfav_plan_t* p, hfav_run_stats* st) {
    if (!p || !st || p->analysis_only) return set_error(HFAV_EINVAL, "bad argument");
    return status(p, st);
}

int hfav_autotune(hfav_plan_t* p, void* const* ax, void* const* go, int n_steps, int reps, void* stream,
                  float* times, int n_times) {
    if (!p || p->analysis_only) return set_error(HFAV_EINVAL, "not an executable plan");
    return autotune(p, ax, go, n_steps, reps, stream, times, n_times);
}

int hfav_plan_timing(hfav_plan_t* p, int enable) {
    if (!p || p->analysis_only) return set_error(HFAV_EINVAL, "not an executable plan");
    return set_timing(p, enable);
}

int hfav_kernel_times(hfav_plan_t* p, char* names, size_t n_names, double* ms, int* counts, int max_kernels) {
    if (!p || !names || !ms || !counts || max_kernels < 1) return set_error(HFAV_EINVAL, "bad argument");
    std::vector<std::string> nm;
    std::vector<double> t;
    std::vector<int> c;
    int rc = kernel_times(p, &nm, &t, &c);
    if (rc) return rc;
    std::string all;
    int k = 0;
    for (; k < (int)nm.size() && k < max_kernels; ++k) {
        all += nm[k] + "\n";
        ms[k] = t[k];
        counts[k] = c[k];
    }
    rc = copy_out(all, names, n_names);
    return rc ? rc : k;
}

void hfav_free(hfav_plan_t* p) {
    if (!p) return;
    destroy_runtime(p);
    delete p;
}

}  // extern "C"
