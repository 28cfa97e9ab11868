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

// fused 2D: the CTA's tile geometry.  A CTA of tx x ty threads owns a tile of
// TX = tx columns and TY = ty x rows_per_thread rows (8 while every field's
// tile fits in 96 KB of shared memory, so two CTAs share an SM, fewer
// otherwise): taller tiles recompute less of the halo.
struct Tile { int hx, hy, w, h; size_t off; };
struct Fused {
    int TX = 0, TY = 0, NT = 0;
    size_t smem = 0;
    std::vector<Tile> tile;
    std::vector<char> inl;      // computed inside its readers, never stored
    std::vector<int> direct;    // goal slot written straight from its rule, else -1
};

int fused_geometry(const hfav_plan_t* p, const Schedule& s, Fused* G) {
    const Dag& d = p->dag;
    const size_t es = p->dtype == HFAV_F64 ? 8 : 4;
    G->TX = s.tx;
    G->NT = s.tx * s.ty;
    G->tile.assign(d.n_fields, Tile());
    std::vector<int> readers(d.n_fields, 0), producer(d.n_fields, -1), goal_slot(d.n_fields, -1);
    std::vector<char> off0(d.n_fields, 1);
    for (size_t r = 0; r < d.rules.size(); ++r) {
        producer[d.rules[r].out[0]] = (int)r;
        for (const hfav_ref& x : d.rules[r].in) {
            readers[x.field]++;
            if (x.off[0] || x.off[1] || x.off[2]) off0[x.field] = 0;
        }
    }
    for (size_t a = 0; a < d.goals.size(); ++a) goal_slot[d.goals[a]] = (int)a;
    auto same = [](const Tile& x, const Tile& y) { return x.hx == y.hx && x.hy == y.hy && x.w == y.w && x.h == y.h; };
    for (int rows = 8; rows >= 1; rows /= 2) {
        G->TY = s.ty * rows;
        for (int f = 0; f < d.n_fields; ++f) {
            // tile of field f over its footprint: [-halo_lo, T + halo_hi) per axis
            const hfav_field_info& fi = p->an.field[f];
            Tile t;
            t.hx = fi.halo_lo[0]; t.hy = fi.halo_lo[1];
            t.w = G->TX + fi.halo_lo[0] + fi.halo_hi[0];
            t.h = G->TY + fi.halo_lo[1] + fi.halo_hi[1];
            t.off = 0;
            G->tile[f] = t;
        }
        // a rule output that every reader takes at offset 0 over the same tile
        // is evaluated inside the readers (a pointwise stage fused into its
        // consumer); a goal that nothing reads, over exactly the tile, is
        // written from its rule to the caller's array
        G->inl.assign(d.n_fields, 0);
        G->direct.assign(d.n_fields, -1);
        for (int f = 0; f < d.n_fields; ++f) {
            const bool produced = producer[f] >= 0 && goal_slot[f] < 0;
            if (produced && readers[f] > 0 && off0[f]) {
                bool ok = true;
                for (const Rule& R : d.rules)
                    for (const hfav_ref& x : R.in)
                        if (x.field == f && !same(G->tile[R.out[0]], G->tile[f])) ok = false;
                G->inl[f] = ok;
            }
            const Tile& t = G->tile[f];
            if (goal_slot[f] >= 0 && producer[f] >= 0 && readers[f] == 0 && t.w == G->TX && t.h == G->TY)
                G->direct[f] = goal_slot[f];
        }
        G->smem = 0;
        for (int f = 0; f < d.n_fields; ++f) {
            if (G->inl[f] || G->direct[f] >= 0) continue;
            G->tile[f].off = G->smem;
            G->smem += ((size_t)G->tile[f].w * G->tile[f].h * es + 15) / 16 * 16;
        }
        if (G->smem <= 96 * 1024) break;
    }
    if (G->smem > 200 * 1024)
        return set_error(HFAV_EUNSUPPORTED, "the fields' tiles exceed shared memory; use a narrower tile");
    // every read of a rule stays inside its input's tile: the footprint of an
    // input covers the footprint of each consumer shifted by the offset
    for (int r : p->an.order) {
        const Rule& R = d.rules[r];
        const Tile& t = G->tile[R.out[0]];
        for (const hfav_ref& x : R.in) {
            const Tile& u = G->tile[x.field];
            const int lo_x = -t.hx + x.off[0], hi_x = t.w - t.hx - 1 + x.off[0];
            const int lo_y = -t.hy + x.off[1], hi_y = t.h - t.hy - 1 + x.off[1];
            if (lo_x < -u.hx || hi_x > u.w - u.hx - 1 || lo_y < -u.hy || hi_y > u.h - u.hy - 1)
                return set_error(HFAV_EINVAL, "internal: a rule's footprint leaves its input's tile");
        }
    }
    return HFAV_OK;
}

// the fused kernel: load the axioms' footprints, evaluate the rules in
// topological order over their own footprints (a barrier between rules), store
// the goals' tiles
std::string fused_source(const hfav_plan_t* p, const Fused& G) {
    const Dag& d = p->dag;
    const int TX = G.TX, TY = G.TY, NT = G.NT;
    // a loop over the w x h cells of a tile, NT threads, unrolled (its trip
    // count is a constant): cell (a, b) of the tile, q = b * w + a
    auto tile_loop = [&](std::ostringstream& c, int w, int h) {
        const int n = w * h, trips = (n + NT - 1) / NT;
        c << "    #pragma unroll\n"
          << "    for (int it = 0; it < " << trips << "; ++it) {\n"
          << "        const int q = tid + it * " << NT << ";\n"
          << "        if (" << (n % NT ? "q < " + std::to_string(n) : std::string("true")) << ") {\n"
          << "        const int a = q % " << w << ", b = q / " << w << ";\n";
    };
    auto direct = [&](int f) { return G.direct[f] >= 0; };
    std::vector<int> producer(d.n_fields, -1);
    for (size_t r = 0; r < d.rules.size(); ++r) producer[d.rules[r].out[0]] = (int)r;
    // the value of field f at the cell (a, b) of tile t shifted by (ox, oy):
    // from f's shared tile, or, for an inlined field, its rule's body on its
    // own inputs at the same cell
    std::function<std::string(int, const Tile&, int, int)> read = [&](int f, const Tile& t, int ox, int oy) {
        if (G.inl[f]) {
            const Rule& R = d.rules[producer[f]];
            std::string v = "hfav_body" + std::to_string(producer[f]) + "(";
            for (size_t k = 0; k < R.in.size(); ++k)
                v += (k ? ", " : "") + read(R.in[k].field, t, R.in[k].off[0], R.in[k].off[1]);
            return v + ")";
        }
        const Tile& u = G.tile[f];
        return "s" + std::to_string(f) + "[(b + " + std::to_string(u.hy - t.hy + oy) + ") * " + std::to_string(u.w) +
               " + (a + " + std::to_string(u.hx - t.hx + ox) + ")]";
    };
    std::ostringstream c;
    c << prelude(p->dtype == HFAV_F64);
    for (int r : p->an.order) c << rule_fn(d.rules[r], "hfav_body" + std::to_string(r));
    c << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") hfav_cg_fused(";
    for (size_t a = 0; a < d.axioms.size(); ++a) c << array_params("x" + std::to_string(a), false) << ", ";
    for (size_t a = 0; a < d.goals.size(); ++a) c << array_params("y" + std::to_string(a), true) << ", ";
    c << "int nx, int ny) {\n"
      << "    extern __shared__ __align__(16) unsigned char smem[];\n"
      << "    const int tid = threadIdx.x, i0 = blockIdx.x * " << TX << ", j0 = blockIdx.y * " << TY << ";\n";
    for (int f = 0; f < d.n_fields; ++f)
        if (!direct(f) && !G.inl[f]) c << "    T* s" << f << " = (T*)(smem + " << G.tile[f].off << ");\n";
    // axioms: the footprint, wrapped (periodic) or from the caller's halo
    for (size_t a = 0; a < d.axioms.size(); ++a) {
        const int f = d.axioms[a];
        const Tile& t = G.tile[f];
        const std::string x = "x" + std::to_string(a);
        tile_loop(c, t.w, t.h);
        c << "        int gi = i0 - " << t.hx << " + a, gj = j0 - " << t.hy << " + b;\n"
          << "        if (" << x << "_w) { gi = hfav_wrap(gi, nx); gj = hfav_wrap(gj, ny); }\n"
          << "        else { gi = min(max(gi, -" << x << "_o0), nx - 1 + " << x << "_o0); gj = min(max(gj, -" << x
          << "_o1), ny - 1 + " << x << "_o1); }\n"
          << "        s" << f << "[q] = " << x << "[(long long)(gj + " << x << "_o1) * " << x << "_p1 + (gi + " << x
          << "_o0)];\n"
          << "    } }\n";
    }
    c << "    __syncthreads();\n";
    for (int r : p->an.order) {
        const Rule& R = d.rules[r];
        const int f = R.out[0];
        if (G.inl[f]) continue;
        const Tile& t = G.tile[f];
        tile_loop(c, t.w, t.h);
        for (size_t k = 0; k < R.in.size(); ++k)
            c << "        const T in" << k << " = " << read(R.in[k].field, t, R.in[k].off[0], R.in[k].off[1]) << ";\n";
        const std::string val = rule_call(R, "hfav_body" + std::to_string(r));
        if (direct(f)) {
            const std::string y = "y" + std::to_string(G.direct[f]);
            c << "        if (i0 + a < nx && j0 + b < ny)\n"
              << "            " << y << "[(long long)(j0 + b + " << y << "_o1) * " << y << "_p1 + (i0 + a + " << y
              << "_o0)] = " << val << ";\n";
        } else {
            c << "        s" << f << "[q] = " << val << ";\n";
        }
        c << "    } }\n";
        c << "    __syncthreads();\n";
    }
    for (size_t a = 0; a < d.goals.size(); ++a) {
        const int f = d.goals[a];
        if (direct(f)) continue;
        const Tile& t = G.tile[f];
        const std::string y = "y" + std::to_string(a);
        tile_loop(c, TX, TY);
        c << "        const int gi = i0 + a, gj = j0 + b;\n"
          << "        if (gi < nx && gj < ny)\n"
          << "            " << y << "[(long long)(gj + " << y << "_o1) * " << y << "_p1 + (gi + " << y << "_o0)] = s" << f
          << "[(b + " << t.hy << ") * " << t.w << " + (a + " << t.hx << ")];\n"
          << "    } }\n";
    }
    c << "}\n";
    return c.str();
}

}  // namespace

int plan_source(const hfav_plan_t* p, std::string* out) {
    if (p->pipeline != PIPE_CODEGEN) return set_error(HFAV_EUNSUPPORTED, "the plan runs no generated kernels");
    if (p->sched.fusion != FUSE_UNFUSED) {
        Fused G;
        int rc = fused_geometry(p, p->sched, &G);
        if (rc) return rc;
        *out = fused_source(p, G);
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
    Fused G;
    int rc = fused_geometry(p, s, &G);
    if (rc) return rc;
    cudaKernel_t k;
    if ((rc = compile(fused_source(p, G), "hfav_cg_fused", &k))) return rc;
    if (G.smem > 48 * 1024)
        HFAV_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G.smem));
    ArgPack A;
    for (size_t a = 0; a < d.axioms.size(); ++a) add_array(A, caller_view_cg(p, ax[a]));
    for (size_t a = 0; a < d.goals.size(); ++a) {
        GArr y = caller_view_cg(p, go[a]);
        y.wrap = 0;
        add_array(A, y);
    }
    const int nx = (int)g.extent[0], ny = (int)g.extent[1];
    A.add(nx);
    A.add(ny);
    auto args = A.ptrs();
    dim3 grd((nx + G.TX - 1) / G.TX, (ny + G.TY - 1) / G.TY);
    HFAV_CUDA(cudaLaunchKernel((const void*)k, grd, dim3(G.NT), args.data(), G.smem, st));
    HFAV_LAUNCHED(p->rt, "codegen_fused", st);
    return HFAV_OK;
}

}  // namespace hfav
