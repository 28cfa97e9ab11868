// codegen.cu -- runtime code generation for rule DAGs that carry user rule
// bodies (HFAV_OP_EXPR): the code generation step of the method (Sec. 3.6:
// with the fusion and storage analysis done, the fused nests are emitted by a
// walk of the nest DAG, each kernel invocation in its phase; Sec. 4.1 leaves
// the emitted scalar loops to a vectorizing compiler), here as CUDA source
// compiled by NVRTC for the device the plan runs on and launched through the
// runtime's library API.
//
// Two forms are generated:
//   * fused (schedule full:smem:TXxTY, 2D DAGs): one kernel per launch; a CTA
//     of TX x TY threads owns a TX-wide tile of the goals, up to 8 TY rows
//     tall; every field gets a shared-memory tile over its footprint (the
//     tile widened by the field's halo from the planner's analysis, Sec.
//     3.5), the axioms are loaded once, and the rules are evaluated in
//     topological order over their footprints, a barrier between rules -- the
//     contraction of every intermediate to a tile, its halo recomputed by the
//     neighbouring tiles;
//   * unfused: one kernel per rule over full arrays (the generic executor's
//     storage) for the EXPR rules of an unfused plan.
// Rule bodies are C expressions over in0 .. in{n-1} (the rule's inputs at
// their offsets) and p0 .. p{m-1} (its parameters, baked in as constants),
// evaluated in the plan's precision inside a device function that sees
// nothing else.  NVRTC is opened at first use, so the library loads on
// machines without it.
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>

#include "common.cuh"

namespace hfav {

namespace {

// ---- NVRTC, opened at first use ---------------------------------------------
struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
    nvrtcResult (*log_size)(nvrtcProgram, size_t*);
    nvrtcResult (*log)(nvrtcProgram, char*);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
    nvrtcResult (*cubin)(nvrtcProgram, char*);
    nvrtcResult (*destroy)(nvrtcProgram*);
};

Nvrtc load_nvrtc() {
    Nvrtc n;
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* nm : names)
        if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) { n.why = "libnvrtc not found"; return n; }
#define SYM(field, name)                                                            \
    n.field = reinterpret_cast<decltype(n.field)>(dlsym(h, name));                 \
    if (!n.field) { n.why = std::string("libnvrtc lacks ") + name; return n; }
    SYM(create, "nvrtcCreateProgram")
    SYM(compile, "nvrtcCompileProgram")
    SYM(log_size, "nvrtcGetProgramLogSize")
    SYM(log, "nvrtcGetProgramLog")
    SYM(cubin_size, "nvrtcGetCUBINSize")
    SYM(cubin, "nvrtcGetCUBIN")
    SYM(destroy, "nvrtcDestroyProgram")
#undef SYM
    n.ok = true;
    return n;
}

Nvrtc& nvrtc() {
    static Nvrtc n = load_nvrtc();
    return n;
}

// compiled kernels by (device, source): generated code depends only on the
// plan's structure, so plans of the same DAG share them
std::mutex g_mu;
std::map<std::string, cudaKernel_t> g_kernels;

int compile(const std::string& src, const char* name, cudaKernel_t* out) {
    int dev = 0;
    HFAV_CUDA(cudaGetDevice(&dev));
    const std::string key = std::to_string(dev) + "\n" + src;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_kernels.find(key);
    if (it != g_kernels.end()) { *out = it->second; return HFAV_OK; }
    Nvrtc& N = nvrtc();
    if (!N.ok) return set_error(HFAV_EUNSUPPORTED, "runtime code generation unavailable: " + N.why);
    int major = 0, minor = 0;
    HFAV_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    HFAV_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor) + "a";
    const char* opts[] = {arch.c_str(), "--std=c++17", "--fmad=true"};
    nvrtcProgram prog;
    if (N.create(&prog, src.c_str(), "hfav_codegen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return set_error(HFAV_ECUDA, "nvrtcCreateProgram failed");
    const nvrtcResult rc = N.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        N.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) N.log(prog, &log[0]);
        N.destroy(&prog);
        return set_error(HFAV_EINVAL, "generated kernel does not compile (check the rule expressions): " + log);
    }
    size_t n = 0;
    N.cubin_size(prog, &n);
    std::string cubin(n, '\0');
    N.cubin(prog, &cubin[0]);
    N.destroy(&prog);
    cudaLibrary_t lib;
    HFAV_CUDA(cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    cudaKernel_t k;
    HFAV_CUDA(cudaLibraryGetKernel(&k, lib, name));
    g_kernels[key] = k;   // the library stays loaded for the life of the process
    *out = k;
    return HFAV_OK;
}

// ---- source pieces -------------------------------------------------------------
std::string lit(double v) {
    char b[64];
    std::snprintf(b, sizeof b, "%.17g", v);
    std::string s = b;
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return "((T)" + s + ")";
}

const char* kPrelude = R"(
__device__ __forceinline__ int hfav_wrap(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    const int r = a % n;
    return r < 0 ? r + n : r;
}
__device__ __forceinline__ T hfav_limflux(T u0, T u1, T l0, T l1) {
    const T f = l1 - l0;
    return f * (u1 - u0) > (T)0 ? (T)0 : f;
}
)";

std::string prelude(bool f64) { return std::string(f64 ? "typedef double T;\n" : "typedef float T;\n") + kPrelude; }

// the rule's value as an expression over in0 .. and its parameters
std::string rule_expr(const Rule& R) {
    std::ostringstream e;
    const int n = (int)R.in.size();
    auto in = [](int k) { return "in" + std::to_string(k); };
    switch (R.op) {
        case HFAV_OP_STENCIL_LINEAR:
            e << "(";
            for (int k = 0; k < n; ++k) e << (k ? " + " : "") << lit(k < (int)R.params.size() ? R.params[k] : 0.0) << " * " << in(k);
            e << ")";
            break;
        case HFAV_OP_GRADMAG_HALF:
            e << "(sqrt(";
            for (int k = 0; k + 1 < n; k += 2)
                e << (k ? " + " : "") << "(" << in(k) << " - " << in(k + 1) << ") * (" << in(k) << " - " << in(k + 1) << ")";
            e << ") * (T)0.5)";
            break;
        case HFAV_OP_SQUASH: e << "(in0 / ((T)1 + in0))"; break;
        case HFAV_OP_LIMFLUX: e << "hfav_limflux(in0, in1, in2, in3)"; break;
        case HFAV_OP_DIFFUSE: e << "(in0 - " << lit(R.params.empty() ? 0.0 : R.params[0]) << " * ((in2 - in1) + (in4 - in3)))"; break;
        default: e << "(" << R.expr << ")"; break;   // HFAV_OP_EXPR
    }
    return e.str();
}

// the rule's body as a device function of its inputs only (the parameters
// p0 .. of an EXPR rule are constants inside): a body sees nothing of the
// kernel around it
std::string rule_fn(const Rule& R, const std::string& name) {
    std::ostringstream o;
    o << "__device__ __forceinline__ T " << name << "(";
    for (size_t k = 0; k < R.in.size(); ++k) o << (k ? ", " : "") << "const T in" << k;
    o << ") {\n";
    if (R.op == HFAV_OP_EXPR)
        for (size_t k = 0; k < R.params.size(); ++k) o << "    const T p" << k << " = " << lit(R.params[k]) << ";\n";
    o << "    return (T)(" << rule_expr(R) << ");\n}\n";
    return o.str();
}

std::string rule_call(const Rule& R, const std::string& name) {
    std::ostringstream o;
    o << name << "(";
    for (size_t k = 0; k < R.in.size(); ++k) o << (k ? ", " : "") << "in" << k;
    o << ")";
    return o.str();
}

// flat kernel arguments, each stored once so the launch can point at it
struct ArgPack {
    std::vector<unsigned char> blob;
    std::vector<size_t> at;
    template <typename V>
    void add(V v) {
        size_t a = (blob.size() + alignof(V) - 1) / alignof(V) * alignof(V);
        blob.resize(a + sizeof(V));
        std::memcpy(&blob[a], &v, sizeof(V));
        at.push_back(a);
    }
    std::vector<void*> ptrs() {
        std::vector<void*> v;
        for (size_t a : at) v.push_back(&blob[a]);
        return v;
    }
};

// the array parameters: pointer, row / plane pitch, origin per axis, extent, wrap
void add_array(ArgPack& A, const GArr& g) {
    A.add((const void*)g.p);
    A.add((long long)g.pitch[1]);
    A.add((long long)g.pitch[2]);
    for (int x = 0; x < 3; ++x) A.add(g.org[x]);
    for (int x = 0; x < 3; ++x) A.add(g.ext[x]);
    A.add(g.wrap);
}

std::string array_params(const std::string& nm, bool out) {
    return std::string(out ? "T* " : "const T* __restrict__ ") + nm + ", long long " + nm + "_p1, long long " + nm +
           "_p2, int " + nm + "_o0, int " + nm + "_o1, int " + nm + "_o2, int " + nm + "_e0, int " + nm + "_e1, int " +
           nm + "_e2, int " + nm + "_w";
}

// view of a caller array of grid 0
GArr caller_view_cg(const hfav_plan_t* p, void* ptr) {
    const hfav_grid& g = p->grids[0];
    GArr a;
    a.p = ptr;
    for (int d = 0; d < 3; ++d) {
        a.pitch[d] = g.pitch[d];
        a.ext[d] = (int)g.extent[d];
        a.org[d] = d < p->dag.ndim ? g.halo : 0;
    }
    a.wrap = p->bc == HFAV_BC_PERIODIC;
    return a;
}

// ---- sources -------------------------------------------------------------------
// unfused: one kernel for one rule.  ref_slot[r] is the input array that
// input r reads (n_slots arrays a0 .. in first-use order); the output array o
// is written over lo .. lo + n - 1.
std::string rule_source(const hfav_plan_t* p, const Rule& R, const std::vector<int>& ref_slot, int n_slots) {
    std::ostringstream s;
    s << prelude(p->dtype == HFAV_F64) << rule_fn(R, "hfav_body")
      << "extern \"C\" __global__ void __launch_bounds__(256) hfav_cg_rule(";
    for (int a = 0; a < n_slots; ++a) s << array_params("a" + std::to_string(a), false) << ", ";
    s << array_params("o", true) << ", int lo0, int lo1, int lo2, int n0, int n1, int n2) {\n"
      << "    const long long total = (long long)n0 * n1 * n2;\n"
      << "    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;\n"
      << "         q += (long long)gridDim.x * blockDim.x) {\n"
      << "        const int i = (int)(q % n0) + lo0;\n"
      << "        const long long rest = q / n0;\n"
      << "        const int j = (int)(rest % n1) + lo1, k = (int)(rest / n1) + lo2;\n";
    for (size_t r = 0; r < R.in.size(); ++r) {
        const std::string a = "a" + std::to_string(ref_slot[r]);
        const hfav_ref& x = R.in[r];
        s << "        T in" << r << ";\n        { int ii = i + (" << x.off[0] << "), jj = j + (" << x.off[1] << "), kk = k + ("
          << x.off[2] << ");\n"
          << "          if (" << a << "_w) { ii = hfav_wrap(ii, " << a << "_e0); jj = hfav_wrap(jj, " << a
          << "_e1); kk = hfav_wrap(kk, " << a << "_e2); }\n"
          << "          in" << r << " = " << a << "[(kk + " << a << "_o2) * " << a << "_p2 + (jj + " << a << "_o1) * " << a
          << "_p1 + (ii + " << a << "_o0)]; }\n";
    }
    s << "        o[(k + o_o2) * o_p2 + (j + o_o1) * o_p1 + (i + o_o0)] = " << rule_call(R, "hfav_body") << ";\n    }\n}\n";
    return s.str();
}

// input arrays of a rule in first-use order: slot of each input
std::vector<int> rule_slots(const Rule& R, std::vector<int>* fields) {
    std::vector<int> slot;
    for (const hfav_ref& x : R.in) {
        auto it = std::find(fields->begin(), fields->end(), x.field);
        slot.push_back((int)(it - fields->begin()));
        if (it == fields->end()) fields->push_back(x.field);
    }
    return slot;
}

// fused 2D: rolling buffers (Sec. 3.5 "Contraction").  A CTA of NT threads
// owns a strip of TXc = NT - (widest footprint in x) columns and a chunk of
// rows, and streams down the chunk one row step at a time.  Every field that
// is read keeps a ring of the last W rows of its strip (its footprint in x)
// in shared memory; a field computed at step s holds row s - lead, its lead
// putting every row it reads in an earlier step, so one barrier per step
// orders the whole DAG.  Axiom rows are fetched P steps ahead with cp.async
// into P extra ring rows.  A stage that all readers take at offset 0 over
// the same footprint is evaluated inside them (never stored); goals go from
// their rule to the caller's arrays.
constexpr int kAhead = 4;   // axiom rows in flight per CTA

struct SField {
    int hxlo = 0, hxhi = 0, hylo = 0, hyhi = 0;
    int w = 0;         // ring row width: TXc + hxlo + hxhi
    int lead = 0;      // computed at step s: row s - lead
    int W = 0;         // ring rows (0: not stored)
    bool axiom = false, inl = false;
    int goal = -1;     // goal slot, -1 if not a goal
    int rule = -1;     // producer
    size_t off = 0;    // shared-memory offset of the ring
    std::vector<std::array<int, 3>> eff;   // (field, dx, dy) read, inlined stages expanded
};
struct Stream {
    int NT = 0, V = 1, TXc = 0, ylo = 0, yhi = 0;   // steps [ylo, jn + yhi)
    int U = 1;                               // steps per unrolled pass
    size_t smem = 0;
    std::vector<SField> f;
};

int stream_geometry_v(const hfav_plan_t* p, const Schedule& s, int V, Stream* S) {
    const Dag& d = p->dag;
    const size_t es = p->dtype == HFAV_F64 ? 8 : 4;
    const int nf = d.n_fields;
    S->NT = s.tx * s.ty;
    S->f.assign(nf, SField());
    std::vector<int> readers(nf, 0);
    std::vector<char> off0(nf, 1);
    for (size_t r = 0; r < d.rules.size(); ++r) {
        S->f[d.rules[r].out[0]].rule = (int)r;
        for (const hfav_ref& x : d.rules[r].in) {
            readers[x.field]++;
            if (x.off[0] || x.off[1] || x.off[2]) off0[x.field] = 0;
        }
    }
    int hxmax = 0;
    for (int f = 0; f < nf; ++f) {
        const hfav_field_info& fi = p->an.field[f];
        SField& F = S->f[f];
        F.hxlo = fi.halo_lo[0]; F.hxhi = fi.halo_hi[0]; F.hylo = fi.halo_lo[1]; F.hyhi = fi.halo_hi[1];
        hxmax = std::max(hxmax, F.hxlo + F.hxhi);
    }
    for (int a : d.axioms) S->f[a].axiom = true;
    for (size_t a = 0; a < d.goals.size(); ++a) S->f[d.goals[a]].goal = (int)a;
    S->V = V;
    S->TXc = S->V * S->NT - hxmax;
    if (S->TXc < 32) return set_error(HFAV_EUNSUPPORTED, "this DAG's footprint is too wide for the tile; use a wider one");
    auto same = [&](int a, int b) {
        const SField &A = S->f[a], &B = S->f[b];
        return A.hxlo == B.hxlo && A.hxhi == B.hxhi && A.hylo == B.hylo && A.hyhi == B.hyhi;
    };
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        F.w = S->TXc + F.hxlo + F.hxhi;
        if (F.rule >= 0 && F.goal < 0 && readers[f] > 0 && off0[f]) {
            bool ok = true;
            for (const Rule& R : d.rules)
                for (const hfav_ref& x : R.in)
                    if (x.field == f && !same(R.out[0], f)) ok = false;
            F.inl = ok;
        }
    }
    // the rows each computed field reads, inlined stages expanded
    std::function<void(int, int, int, std::vector<std::array<int, 3>>*)> expand =
        [&](int f, int dx, int dy, std::vector<std::array<int, 3>>* out) {
            for (const hfav_ref& x : d.rules[S->f[f].rule].in) {
                if (S->f[x.field].inl) expand(x.field, dx + x.off[0], dy + x.off[1], out);
                else out->push_back({x.field, dx + x.off[0], dy + x.off[1]});
            }
        };
    for (int r : p->an.order) {
        const int f = d.rules[r].out[0];
        SField& F = S->f[f];
        if (F.inl) continue;
        expand(f, 0, 0, &F.eff);
        int lead = -(1 << 20);
        for (auto& e : F.eff) lead = std::max(lead, S->f[e[0]].lead + e[2]);
        F.lead = lead + 1;
    }
    // ring rows: from the oldest row a reader still needs to the newest written
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        if (F.inl) continue;
        for (int c = 0; c < nf; ++c)
            for (auto& e : S->f[c].eff)
                if (e[0] == f) F.W = std::max(F.W, S->f[c].lead - F.lead - e[2] + 1);
        if (F.axiom) F.W = std::max(F.W, 1) + kAhead;
        // a power of two, so that one unrolled pass of U = max W steps sees
        // every ring at fixed rows
        if (F.W > 0) { int w2 = 1; while (w2 < F.W) w2 *= 2; F.W = w2; }
        S->U = std::max(S->U, F.W);
    }
    S->smem = 0;
    S->ylo = 1 << 20;
    S->yhi = -(1 << 20);
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        if (F.inl) continue;
        if (F.W > 0) {
            F.off = S->smem;
            S->smem += ((size_t)F.W * F.w * es + 15) / 16 * 16;
        }
        if (F.axiom || F.rule >= 0) {
            S->ylo = std::min(S->ylo, -F.hylo + F.lead);
            S->yhi = std::max(S->yhi, F.hyhi + F.lead);
        }
    }
    if (S->smem > 200 * 1024) return set_error(HFAV_EUNSUPPORTED, "the fields' rings exceed shared memory");
    // every read stays inside the ring it reads: columns within the input's
    // footprint, rows within its footprint and still in the ring
    for (int f = 0; f < nf; ++f) {
        const SField& F = S->f[f];
        if (F.inl || F.rule < 0) continue;
        for (auto& e : F.eff) {
            const SField& G = S->f[e[0]];
            const bool cols = -F.hxlo + e[1] >= -G.hxlo && F.hxhi + e[1] <= G.hxhi;
            const bool rows = -F.hylo + e[2] >= -G.hylo && F.hyhi + e[2] <= G.hyhi;
            const bool ring = F.lead - G.lead - e[2] >= 1 && F.lead - G.lead - e[2] + 1 <= G.W - (G.axiom ? kAhead : 0);
            if (!cols || !rows || !ring) return set_error(HFAV_EINVAL, "internal: a rule reads outside its input's ring");
        }
    }
    return HFAV_OK;
}

// each thread takes V columns of a row (tid, tid + NT, ...): the per-step
// work (row checks, fetch set-up, barrier) is shared by V cells.  V = 4 (FP32)
// or 2 (FP64), halved while the rings need more than 96 KB of shared memory.
int stream_geometry(const hfav_plan_t* p, const Schedule& s, Stream* S) {
    int rc = HFAV_EUNSUPPORTED;
    for (int V = p->dtype == HFAV_F64 ? 2 : 4; V >= 1; V /= 2) {
        *S = Stream();
        rc = stream_geometry_v(p, s, V, S);
        if (rc == HFAV_OK && S->smem <= 96 * 1024) return HFAV_OK;
    }
    return rc;
}

std::string stream_source(const hfav_plan_t* p, const Stream& S) {
    const Dag& d = p->dag;
    const bool f64 = p->dtype == HFAV_F64;
    const int NT = S.NT, TXc = S.TXc;
    auto slot = [](const std::string& row, int W) {   // ring row of a (possibly negative) row index
        return "((unsigned)(" + row + " + " + std::to_string(1024 * W) + ") % " + std::to_string(W) + "u)";
    };
    std::ostringstream c;
    c << prelude(f64)
      << "__device__ __forceinline__ void hfav_cp(void* dst, const void* src) {\n"
      << "    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);\n"
      << "    asm volatile(\"cp.async.ca.shared.global [%0], [%1], " << (f64 ? 8 : 4)
      << ";\\n\" :: \"r\"(sa), \"l\"(src) : \"memory\");\n"
      << "}\n"
      << "__device__ __forceinline__ void hfav_commit() { asm volatile(\"cp.async.commit_group;\\n\" ::: \"memory\"); }\n"
      << "__device__ __forceinline__ void hfav_wait() { asm volatile(\"cp.async.wait_group " << kAhead
      << ";\\n\" ::: \"memory\"); }\n";
    for (int r : p->an.order) c << rule_fn(d.rules[r], "hfav_body" + std::to_string(r));
    c << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") hfav_cg_fused(";
    for (size_t a = 0; a < d.axioms.size(); ++a) c << array_params("x" + std::to_string(a), false) << ", ";
    for (size_t a = 0; a < d.goals.size(); ++a) c << array_params("y" + std::to_string(a), true) << ", ";
    c << "int nx, int ny, int CH) {\n"
      << "    extern __shared__ __align__(16) unsigned char smem[];\n"
      << "    const int tid = threadIdx.x, i0 = blockIdx.x * " << TXc << ", j0 = blockIdx.y * CH;\n"
      << "    const int jn = min(CH, ny - j0);\n";
    for (int f = 0; f < d.n_fields; ++f)
        if (!S.f[f].inl && S.f[f].W > 0) c << "    T* s" << f << " = (T*)(smem + " << S.f[f].off << ");\n";
    // a thread's columns tid + v NT, v < V, of a ring row of width w: the
    // condition that column set v is inside ("" when always, "-" never)
    const int V = S.V;
    auto inside = [&](int v, int w) -> std::string {
        if (w - v * NT >= NT) return "";
        if (w - v * NT <= 0) return "-";
        return "tid < " + std::to_string(w - v * NT);
    };
    // axioms: each thread's columns (fixed), a row fetch issued kAhead steps ahead
    for (size_t a = 0; a < d.axioms.size(); ++a) {
        const int f = d.axioms[a];
        const SField& F = S.f[f];
        const std::string x = "x" + std::to_string(a);
        for (int v = 0; v < V; ++v) {
            const std::string cv = std::to_string(a) + "_" + std::to_string(v);
            if (inside(v, F.w) == "-") continue;
            c << "    int col" << cv << " = i0 - " << F.hxlo << " + tid + " << v * NT << ";\n"
              << "    if (" << x << "_w) col" << cv << " = hfav_wrap(col" << cv << ", nx);\n"
              << "    else col" << cv << " = min(max(col" << cv << ", -" << x << "_o0), nx - 1 + " << x << "_o0);\n"
              << "    const T* src" << cv << " = " << x << " + col" << cv << " + " << x << "_o0;\n";
        }
        c << "    auto fetch" << a << " = [&](int r) {\n"
          << "        if (r >= -" << F.hylo << " && r < jn + " << F.hyhi << ") {\n"
          << "            int gj = j0 + r;\n"
          << "            if (" << x << "_w) gj = hfav_wrap(gj, ny);\n"
          << "            else gj = min(max(gj, -" << x << "_o1), ny - 1 + " << x << "_o1);\n"
          << "            const long long ro = (long long)(gj + " << x << "_o1) * " << x << "_p1;\n"
          << "            T* const dst = s" << f << " + " << slot("r", F.W) << " * " << F.w << " + tid;\n";
        for (int v = 0; v < V; ++v) {
            const std::string in = inside(v, F.w), cv = std::to_string(a) + "_" + std::to_string(v);
            if (in == "-") continue;
            c << "            " << (in.empty() ? "" : "if (" + in + ") ") << "hfav_cp(dst + " << v * NT << ", src" << cv
              << " + ro);\n";
        }
        c << "        }\n"
          << "    };\n";
    }
    for (int f = 0; f < d.n_fields; ++f) {
        const SField& F = S.f[f];
        if (F.goal < 0) continue;
        const std::string y = "y" + std::to_string(F.goal);
        for (int v = 0; v < V; ++v) {
            const std::string g = std::to_string(F.goal) + "_" + std::to_string(v);
            if (inside(v, F.w) == "-") continue;
            c << "    const int gx" << g << " = tid + " << v * NT - F.hxlo << ";\n"
              << "    const bool gok" << g << " = gx" << g << " >= 0 && gx" << g << " < " << TXc << " && i0 + gx" << g
              << " < nx;\n"
              << "    T* const gcol" << g << " = " << y << " + (long long)" << y << "_o1 * " << y << "_p1 + (i0 + gx"
              << g << " + " << y << "_o0);\n";
        }
    }
    c << "    #pragma unroll 1\n"
      << "    for (int r = " << S.ylo << "; r < " << S.ylo + kAhead << "; ++r) {\n";
    for (size_t a = 0; a < d.axioms.size(); ++a) c << "        fetch" << a << "(r);\n";
    c << "        hfav_commit();\n    }\n";
    // the step loop in passes of U steps: step s = sp + k with sp - ylo a
    // multiple of U, so the ring row of row sp + k - lead + dy is a constant
    const int U = S.U;
    auto cslot = [&](int k, int lead, int dy, int W) { return ((S.ylo + k - lead + dy) % W + W) % W; };
    c << "    #pragma unroll 1\n"
      << "    for (int sp = " << S.ylo << "; sp < jn + " << S.yhi << "; sp += " << U << ") {\n";
    for (int k = 0; k < U; ++k) {
        c << "    {   // step sp + " << k << "\n"
          << "        const int s = sp + " << k << ";\n";
        for (size_t a = 0; a < d.axioms.size(); ++a) c << "        fetch" << a << "(s + " << kAhead << ");\n";
        c << "        hfav_commit();\n";
        for (int r : p->an.order) {
            const Rule& R = d.rules[r];
            const int f = R.out[0];
            const SField& F = S.f[f];
            if (F.inl) continue;
            c << "        {\n"
              << "            const int r = s - " << F.lead << ";\n"
              << "            if (r >= -" << F.hylo << " && r < jn + " << F.hyhi << ") {\n";
            for (int v = 0; v < V; ++v) {
                const std::string in = inside(v, F.w);
                if (in == "-") continue;
                // the value of field g at this thread's cell (column set v) shifted by (dx, dy)
                std::function<std::string(int, int, int)> read = [&](int g, int dx, int dy) -> std::string {
                    const SField& G = S.f[g];
                    if (G.inl) {
                        const Rule& Q = d.rules[G.rule];
                        std::string val = "hfav_body" + std::to_string(G.rule) + "(";
                        for (size_t q = 0; q < Q.in.size(); ++q)
                            val += (q ? ", " : "") + read(Q.in[q].field, dx + Q.in[q].off[0], dy + Q.in[q].off[1]);
                        return val + ")";
                    }
                    return "s" + std::to_string(g) + "[" +
                           std::to_string(cslot(k, F.lead, dy, G.W) * G.w + dx + G.hxlo - F.hxlo + v * NT) + " + tid]";
                };
                c << "            " << (in.empty() ? "{" : "if (" + in + ") {") << "\n";
                for (size_t q = 0; q < R.in.size(); ++q)
                    c << "                const T in" << q << " = " << read(R.in[q].field, R.in[q].off[0], R.in[q].off[1])
                      << ";\n";
                c << "                const T v = " << rule_call(R, "hfav_body" + std::to_string(r)) << ";\n";
                if (F.W > 0)
                    c << "                s" << f << "[" << cslot(k, F.lead, 0, F.W) * F.w + v * NT << " + tid] = v;\n";
                if (F.goal >= 0) {
                    const std::string g = std::to_string(F.goal) + "_" + std::to_string(v);
                    c << "                if (r >= 0 && r < jn && gok" << g << ")\n"
                      << "                    gcol" << g << "[(long long)(j0 + r) * y" << F.goal << "_p1] = v;\n";
                }
                c << "            }\n";
            }
            c << "            }\n        }\n";
        }
        c << "        hfav_wait();\n"
          << "        __syncthreads();\n"
          << "    }\n";
    }
    c << "    }\n"
      << "    asm volatile(\"cp.async.wait_all;\\n\" ::: \"memory\");\n"
      << "}\n";
    return c.str();
}

}  // namespace

int plan_source(const hfav_plan_t* p, std::string* out) {
    if (p->pipeline != PIPE_CODEGEN) return set_error(HFAV_EUNSUPPORTED, "the plan runs no generated kernels");
    if (p->sched.fusion != FUSE_UNFUSED) {
        Stream S;
        int rc = stream_geometry(p, p->sched, &S);
        if (rc) return rc;
        *out = stream_source(p, S);
        return HFAV_OK;
    }
    std::ostringstream o;
    for (int r : p->an.order) {
        const Rule& R = p->dag.rules[r];
        if (R.op != HFAV_OP_EXPR) continue;
        std::vector<int> fields;
        const std::vector<int> slot = rule_slots(R, &fields);
        o << "// ---- rule " << r << "\n" << rule_source(p, R, slot, (int)fields.size());
    }
    *out = o.str();
    return HFAV_OK;
}

// ---- launchers -------------------------------------------------------------------
int launch_cg_rule(hfav_plan_t* p, const Rule& R, const std::vector<int>& ref_slot, const std::vector<GArr>& ins,
                   const GArr& out, const int* lo, const int* n, cudaStream_t st) {
    cudaKernel_t k;
    int rc = compile(rule_source(p, R, ref_slot, (int)ins.size()), "hfav_cg_rule", &k);
    if (rc) return rc;
    ArgPack A;
    for (auto& g : ins) add_array(A, g);
    add_array(A, out);
    for (int x = 0; x < 3; ++x) A.add(lo[x]);
    for (int x = 0; x < 3; ++x) A.add(n[x]);
    auto args = A.ptrs();
    const int64_t total = (int64_t)n[0] * n[1] * n[2];
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
    HFAV_CUDA(cudaLaunchKernel((const void*)k, dim3(blocks), dim3(256), args.data(), 0, st));
    HFAV_LAUNCHED(p->rt, "codegen_rule", st);
    return HFAV_OK;
}

int launch_codegen(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st) {
    if (s.fusion == FUSE_UNFUSED) return launch_generic(p, ax, go, st);
    const Dag& d = p->dag;
    const hfav_grid& g = p->grids[0];
    Stream S;
    int rc = stream_geometry(p, s, &S);
    if (rc) return rc;
    cudaKernel_t k;
    if ((rc = compile(stream_source(p, S), "hfav_cg_fused", &k))) return rc;
    if (S.smem > 48 * 1024)
        HFAV_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem));
    const int nx = (int)g.extent[0], ny = (int)g.extent[1];
    // rows per chunk: the wave count that costs least, each chunk paying the
    // pipeline's fill (yhi - ylo steps beyond its rows)
    int dev = 0, sms = 0, per_sm = 0;
    HFAV_CUDA(cudaGetDevice(&dev));
    HFAV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, S.NT, S.smem));
    const int64_t resident = (int64_t)std::max(1, sms) * std::max(1, per_sm);
    const int64_t strips = (nx + S.TXc - 1) / S.TXc;
    const int fill = S.yhi - S.ylo;
    int CH = ny;
    double best = 1e300;
    for (int64_t chunks = 1; chunks <= ny; chunks = chunks < 8 ? chunks + 1 : chunks * 5 / 4) {
        const int ch = (int)((ny + chunks - 1) / chunks);
        const int64_t ctas = strips * ((ny + ch - 1) / ch);
        const double cost = (double)(ch + fill) * (double)((ctas + resident - 1) / resident);
        if (cost < best) { best = cost; CH = ch; }
    }
    ArgPack A;
    for (size_t a = 0; a < d.axioms.size(); ++a) add_array(A, caller_view_cg(p, ax[a]));
    for (size_t a = 0; a < d.goals.size(); ++a) {
        GArr y = caller_view_cg(p, go[a]);
        y.wrap = 0;
        add_array(A, y);
    }
    A.add(nx);
    A.add(ny);
    A.add(CH);
    auto args = A.ptrs();
    dim3 grd((unsigned)strips, (unsigned)((ny + CH - 1) / CH));
    HFAV_CUDA(cudaLaunchKernel((const void*)k, grd, dim3(S.NT), args.data(), S.smem, st));
    HFAV_LAUNCHED(p->rt, "codegen_fused", st);
    return HFAV_OK;
}

}  // namespace hfav
