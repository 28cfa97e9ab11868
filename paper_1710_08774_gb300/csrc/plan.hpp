// plan.hpp -- internal plan object shared by the planner, the runtime and the
// kernel launchers of libhfav.so (never installed; the public ABI is hfav.h).
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <memory>
#include <vector>

#include "../../include/hfav.h"

namespace hfav {

struct Rule {
    int op = 0;
    int axis = 0;
    std::vector<hfav_ref> in;
    std::vector<int> out;
    std::vector<double> params;
    std::string expr;   // HFAV_OP_EXPR body
};

struct Dag {
    int n_fields = 0;
    std::vector<int> rank;
    std::vector<Rule> rules;
    std::vector<int> axioms, goals;
    int ndim = 2;
    int stream_axis = 1;
    int feedback = 0;
    std::vector<int> inout;   // per goal: index of the axiom it may alias, -1 for none
};

// Schedule axes: fusion x placement x tile (the variant space of the cost model).
enum Fusion { FUSE_FULL = 0, FUSE_SWEEP = 1, FUSE_UNFUSED = 2 };
enum Placement { PLACE_REG = 0, PLACE_SMEM = 1, PLACE_HBM = 2 };

struct Schedule {
    int fusion = FUSE_FULL;
    int placement = PLACE_REG;
    int tx = 32, ty = 4;
    std::string str() const;
};

bool parse_schedule(const char* s, Schedule* out, std::string* err);

// Kernel pipelines the planner can map a fusion group onto.
enum Pipeline { PIPE_GENERIC = 0, PIPE_CHAIN2D = 1, PIPE_CHAIN3D = 2, PIPE_GODUNOV = 3, PIPE_COSMO = 4, PIPE_CODEGEN = 5 };

// Field ids of a recognised Godunov DAG (x sweep then y sweep, optional CFL).
struct GodunovMap {
    double gamma = 1.4, cfl = 0.5;
    int newton_max = 10;          // RIEMANN params[1] when given: cap on Newton iterations (1..10)
    int cfl_rule = -1;
    int sweep_rules[2][8] = {};   // rule ids per axis in kernel order
};

// Rule ids / weights of a recognised stencil chain.
struct ChainMap {
    double w1[27] = {};   // first linear stencil, 3x3(x3) box weights, index (dk+1)*9+(dj+1)*3+(di+1)
    double w2[27] = {};   // second linear stencil (3D chain only)
    double coef = 0.0;    // COSMO: diffusion coefficient c of ustage
    int rules[4] = {-1, -1, -1, -1};
};

struct Runtime;   // device-side state (runtime.cu)

// Analysis results (Sec. 3.2 - 3.5).
struct Analysis {
    std::vector<int> order;          // topological rule order
    std::vector<int> rule_group;     // fusion group per rule
    int n_groups = 0;
    std::vector<hfav_field_info> field;
    std::vector<int> group_rank;     // iteration rank (irank) of each group's nest
    int max_depth = 0;               // longest rule chain
    int max_radius = 0;              // largest |offset| over all refs
};

}  // namespace hfav

struct hfav_plan_s {
    hfav::Dag dag;
    std::vector<hfav_grid> grids;
    int dtype = HFAV_F64;
    int bc = HFAV_BC_PERIODIC;
    bool analysis_only = false;
    hfav::Analysis an;
    int pipeline = hfav::PIPE_GENERIC;
    hfav::GodunovMap gmap;
    hfav::ChainMap cmap;
    hfav::Schedule sched;
    bool tune_first_run = false;   // schedule "tuned": autotune on the first run's arrays
    hfav::Runtime* rt = nullptr;
    std::shared_ptr<void> cg_cache;   // generated kernels prepared per schedule (codegen.cu)
};

namespace hfav {
// planner.cpp
int copy_dag(const hfav_dag* in, Dag* out);
int analyze(hfav_plan_t* p, const int64_t* extent);
int recognise(hfav_plan_t* p);
std::vector<Schedule> valid_schedules(const hfav_plan_t* p);
bool schedule_valid(const hfav_plan_t* p, const Schedule& s, std::string* why);
std::string dump_json(const hfav_plan_t* p);
void features(const hfav_plan_t* p, const Schedule& s, float* f);

// errors.cpp-style helpers (api.cpp)
int set_error(int code, const std::string& msg);

// codegen.cu: the CUDA source a plan of generated kernels compiles; whether
// a schedule updates declared in/out pairs in place (no full snapshot)
int plan_source(const hfav_plan_t* p, std::string* out);
bool codegen_inplace(const hfav_plan_t* p, const Schedule& s);
// the generated warp-strip kernel (full:reg) applies to the plan's DAG and tile
bool codegen_wstrip_ok(const hfav_plan_t* p, const Schedule& s, std::string* why);

// runtime.cu
int run(hfav_plan_t* p, void* const* ax, void* const* go, int n_steps, void* stream, bool graph);
int status(hfav_plan_t* p, hfav_run_stats* st);
int autotune(hfav_plan_t* p, void* const* ax, void* const* go, int n_steps, int reps, void* stream,
             float* times, int n_times);
void destroy_runtime(hfav_plan_t* p);
void drop_graph(hfav_plan_t* p);
int kernel_times(hfav_plan_t* p, std::vector<std::string>* names, std::vector<double>* ms, std::vector<int>* counts);
int set_timing(hfav_plan_t* p, int on);
// resident warps per SM of a schedule's main kernel (-1 without a device)
double chain_kernel_warps(const hfav_plan_t* p, const Schedule& s);
double godunov_kernel_warps(const hfav_plan_t* p, const Schedule& s);
}  // namespace hfav
