// codegen.cu -- runtime code generation for rule DAGs with user rule bodies
// (HFAV_OP_EXPR), reductions to scalars, or declared in/out aliasing: the code
// generation step of the method (Sec. 3.6: with the fusion and storage
// analysis done, the fused nests are emitted by a walk of the nest DAG, each
// kernel invocation in its phase; Sec. 4.1 leaves the emitted scalar loops to
// a vectorizing compiler), here as CUDA source compiled by NVRTC for the
// device the plan runs on and launched through the runtime's library API.
//
// What is generated (details at each generator below):
//   * fused 2D plans: one kernel per fusion group of the analysis -- a
//     streaming kernel whose fields live in rolling row rings in shared memory
//     (Sec. 3.5 "Contraction"), or, for a group without offsets, a pointwise
//     kernel in registers; reductions accumulate inside the group that
//     produces their input and a one-CTA finalization combines them (Sec. 3.4);
//   * unfused plans: one kernel per rule;
//   * in-place runs of declared in/out pairs: two small kernels that save the
//     halo bands the streaming kernel cannot read live.
// Rule bodies are C expressions over in0 .. in{n-1} (the rule's inputs at
// their offsets) and p0 .. p{m-1} (its parameters, baked in as constants),
// evaluated in the plan's precision inside a device function that sees
// nothing else.  NVRTC is opened at first use, so the library loads on
// machines without it.
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <mutex>
#include <sstream>

#include "common.cuh"

namespace hfav {

// The halo bands an in-place streaming kernel cannot read live (Sec. 3.5 "In/
// out chaining": the input values still needed are copied to temporaries
// before the outputs overwrite them).  For strip b (columns i0 = b TXc ..,
// interior width wint = min(TXc, nx - i0)) the column band holds, for every
// row g in [-hylo, ny + hyhi), the hxlo columns left of the interior and the
// hxhi right of it; for chunk c (rows j0 = c CH .., jn = min(CH, ny - j0))
// the row band holds the hylo rows above and the hyhi below, over all columns
// [-hxlo, nx + hxhi).  Indices wrap (periodic) or clamp into the caller's halo
// exactly as the kernel's own fetches do.  HXa, HYa: band widths, at least 1.
// Two kernels, one per band, with no division per element.
template <typename T>
__device__ __forceinline__ T band_load(const GArr& src, int gi, int gj, int nx, int ny) {
    if (!src.wrap) {
        gi = min(max(gi, -src.org[0]), nx - 1 + src.org[0]);
        gj = min(max(gj, -src.org[1]), ny - 1 + src.org[1]);
    }
    return garr_ld<T>(src, gi, gj, 0);
}

// column bands: one thread per (strip, row), its HXa columns
template <typename T>
__global__ void __launch_bounds__(256) inout_colband(const GArr src, T* __restrict__ cb, int nx, int ny, int TXc,
                                                     int hxlo, int hylo, int rows, int HXa, int pairs) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= pairs) return;
    const int b = q / rows, g = q - b * rows - hylo;
    const int i0 = b * TXc, wint = min(TXc, nx - i0);
    for (int k = 0; k < HXa; ++k) {
        const int x = k < hxlo ? k - hxlo : wint + (k - hxlo);
        cb[(int64_t)q * HXa + k] = band_load<T>(src, i0 + x, g, nx, ny);
    }
}

// row bands: blockIdx.y = (chunk, band row), threads along the columns
template <typename T>
__global__ void __launch_bounds__(256) inout_rowband(const GArr src, T* __restrict__ rb, int nx, int ny, int CH,
                                                     int hxlo, int hylo, int cols, int HYa) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    const int c = blockIdx.y / HYa, k = blockIdx.y - c * HYa;
    const int j0 = c * CH, jn = min(CH, ny - j0);
    const int r = k < hylo ? k - hylo : jn + (k - hylo);
    rb[(int64_t)blockIdx.y * cols + col] = band_load<T>(src, col - hxlo, j0 + r, nx, ny);
}

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
// a parameter as a literal of the plan's type: 17 significant digits restore
// any finite double exactly; infinities and NaNs (no C spelling) by their bits
std::string lit(double v) {
    char b[64];
    if (!std::isfinite(v)) {
        unsigned long long bits;
        std::memcpy(&bits, &v, sizeof bits);
        std::snprintf(b, sizeof b, "__longlong_as_double(0x%016llxULL)", bits);
        return "((T)" + std::string(b) + ")";
    }
    std::snprintf(b, sizeof b, "%.17g", v);
    std::string s = b;
    if (s.find_first_of(".eE") == std::string::npos) s += ".0";
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
        case HFAV_OP_REDUCE_SUM: case HFAV_OP_REDUCE_MAX: e << "in0"; break;   // the value reduced
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

// Fused 2D: rolling buffers (Sec. 3.5 "Contraction").  A streaming kernel
// evaluates a part of the DAG: a fusion group of the analysis (the fused
// form) or one rule (the unfused form of DAGs with reductions).  A CTA of NT
// threads owns a strip of TXc = V NT - (widest footprint in x) columns, V
// columns per thread, and a chunk of rows, and streams down the chunk one row
// step at a time.  Every field the part reads keeps a ring of the last W rows
// of its strip (its footprint in x) in shared memory; a field computed at
// step s holds row s - lead, its lead putting every row it reads in an
// earlier step, so one barrier per step orders the part.  Rows of the fields
// the part reads from memory arrive P steps ahead by cp.async into P extra
// ring rows.  A stage that all its readers take at offset 0 over the same
// footprint is evaluated inside them (never stored).
//
// Reductions (Sec. 3.4) accumulate over the interior in the part that
// produces their input (the steady state), one FP64 partial per CTA; a
// one-CTA kernel then combines the partials in a fixed order and evaluates
// the scalar rules (the finalization), and later parts read the scalars (the
// broadcast).  Fields that cross from one part to a later one (the split)
// are full arrays over their footprint.
constexpr int kAhead = 4;   // rows in flight per CTA for the fields read from memory

struct Part {
    std::vector<int> rules;   // grid rules and reductions, topological order
};

// A reduction's per-thread accumulator.  FP64 plans add in FP64.  FP32 plans
// keep an FP32 sum with Neumaier's compensation (Neumaier 1974, the improved
// Kahan-Babuska summation: a second FP32 term collects each addition's
// rounding error) -- FP64 adds run at a small fraction of the FP32 rate on
// this part -- and the maximum in FP32 (exact); each thread's result then
// joins the CTA's FP64 partial.
std::string red_decl(int k, bool mx, bool f64) {
    const std::string K = std::to_string(k);
    if (mx) return "    T racc" + K + " = (T)__longlong_as_double(0xfff0000000000000ULL);\n";
    if (f64) return "    double racc" + K + " = 0.0;\n";
    return "    float racc" + K + " = 0.f, rcmp" + K + " = 0.f;\n";
}
std::string red_add(int k, bool mx, bool f64, const std::string& x) {
    const std::string K = std::to_string(k), a = "racc" + K;
    if (mx) return a + " = fmax(" + a + ", " + x + ");";
    if (f64) return a + " = " + a + " + " + x + ";";
    return "{ const float hx = " + x + ", ht = " + a + " + hx; rcmp" + K + " += fabsf(" + a + ") >= fabsf(hx) ? (" + a +
           " - ht) + hx : (hx - ht) + " + a + "; " + a + " = ht; }";
}
std::string red_final(int k, bool mx, bool f64) {
    const std::string K = std::to_string(k);
    if (mx || f64) return "(double)racc" + K;
    return "((double)racc" + K + " + (double)rcmp" + K + ")";
}

struct SField {
    int hxlo = 0, hxhi = 0, hylo = 0, hyhi = 0;
    int w = 0;          // ring row width: TXc + hxlo + hxhi
    int lead = 0;       // computed at step s: row s - lead
    int W = 0;          // ring rows (0: not stored)
    bool scalar = false, inl = false;
    int load = -1;      // kernel array it is read from (x<load>), -1 if computed here or unused
    int goal = -1;      // caller goal array it is written to (y<goal>, interior)
    int cross = -1;     // plan array it is written to (z<cross>, owned cells of its footprint)
    int red = -1;       // reduction slot: the part's reduction writing this rank-0 field
    int rule = -1;      // producer inside the part
    size_t off = 0;     // shared-memory offset of the ring
    std::vector<std::array<int, 3>> eff;   // (field, dx, dy) read, inlined stages expanded
};

struct Stream {
    bool pointwise = false;                          // no offsets, no halos: no rings
    int NT = 0, V = 1, TXc = 0, ylo = 0, yhi = 0;   // steps [ylo, jn + yhi)
    int U = 1;                                      // steps per unrolled pass
    size_t smem = 0;
    std::vector<SField> f;
    std::vector<int> loads, goals, crosses, reds, scalars;   // fields, in parameter / slot order
    std::vector<int> goal_slot;                              // caller goal index of each goals[k]
    std::vector<char> inplace;                               // per load: its array is also written (in/out)
};

bool in_part(const Part& P, int r) { return std::find(P.rules.begin(), P.rules.end(), r) != P.rules.end(); }

int stream_geometry_v(const hfav_plan_t* p, const Schedule& s, const Part& P, int V, Stream* S) {
    const Dag& d = p->dag;
    const size_t es = p->dtype == HFAV_F64 ? 8 : 4;
    const int nf = d.n_fields;
    S->NT = s.tx * s.ty;
    S->V = V;
    S->f.assign(nf, SField());
    std::vector<int> readers(nf, 0);
    std::vector<char> off0(nf, 1), outside(nf, 0), involved(nf, 0);
    for (size_t r = 0; r < d.rules.size(); ++r) {
        const bool mine = in_part(P, (int)r);
        for (const hfav_ref& x : d.rules[r].in) {
            if (!mine) { outside[x.field] = 1; continue; }
            readers[x.field]++;
            involved[x.field] = 1;
            if (x.off[0] || x.off[1] || x.off[2]) off0[x.field] = 0;
        }
    }
    for (int r : P.rules) { S->f[d.rules[r].out[0]].rule = r; involved[d.rules[r].out[0]] = 1; }
    int hxmax = 0;
    for (int f = 0; f < nf; ++f) {
        const hfav_field_info& fi = p->an.field[f];
        SField& F = S->f[f];
        F.scalar = d.rank[f] == 0;
        F.hxlo = fi.halo_lo[0]; F.hxhi = fi.halo_hi[0]; F.hylo = fi.halo_lo[1]; F.hyhi = fi.halo_hi[1];
        if (involved[f]) hxmax = std::max(hxmax, F.hxlo + F.hxhi);
    }
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        if (!involved[f]) continue;
        if (F.scalar) {
            if (F.rule >= 0) { F.red = (int)S->reds.size(); S->reds.push_back(f); }
            else if (readers[f]) S->scalars.push_back(f);
            continue;
        }
        if (F.rule < 0) { F.load = (int)S->loads.size(); S->loads.push_back(f); continue; }
        const auto g = std::find(d.goals.begin(), d.goals.end(), f);
        if (g != d.goals.end()) {
            F.goal = (int)S->goals.size();
            S->goals.push_back(f);
            S->goal_slot.push_back((int)(g - d.goals.begin()));
        }
        if (outside[f]) { F.cross = (int)S->crosses.size(); S->crosses.push_back(f); }
    }
    // a pointwise part (every read at offset 0, every field without a halo)
    // needs no rings: each cell is loaded, computed and stored in registers
    bool pw = hxmax == 0;
    for (int f = 0; f < nf; ++f)
        if (involved[f] && (S->f[f].hylo || S->f[f].hyhi || (!S->f[f].scalar && !off0[f] && readers[f]))) pw = false;
    if (pw) {
        S->inplace.assign(S->loads.size(), 0);
        S->pointwise = true;
        S->TXc = S->V * S->NT;
        for (int f = 0; f < nf; ++f) {
            SField& F = S->f[f];
            F.w = S->TXc;
            F.inl = F.rule >= 0 && !F.scalar && F.goal < 0 && F.cross < 0;   // every stored value goes to memory
        }
        return HFAV_OK;
    }
    S->inplace.assign(S->loads.size(), 0);
    S->TXc = S->V * S->NT - hxmax;
    if (S->TXc < 32) return set_error(HFAV_EUNSUPPORTED, "this DAG's footprint is too wide for the tile; use a wider one");
    auto same = [&](int a, int b) {
        const SField &A = S->f[a], &B = S->f[b];
        return A.hxlo == B.hxlo && A.hxhi == B.hxhi && A.hylo == B.hylo && A.hyhi == B.hyhi;
    };
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        F.w = S->TXc + F.hxlo + F.hxhi;
        if (F.rule >= 0 && !F.scalar && F.goal < 0 && F.cross < 0 && readers[f] > 0 && off0[f]) {
            bool ok = true;
            for (int r : P.rules)
                for (const hfav_ref& x : d.rules[r].in)
                    if (x.field == f && !same(d.rules[r].out[0], f)) ok = false;
            F.inl = ok;
        }
    }
    // the rows each computed field reads, inlined stages expanded (scalars are
    // kernel constants, not rows)
    std::function<void(int, int, int, std::vector<std::array<int, 3>>*)> expand =
        [&](int f, int dx, int dy, std::vector<std::array<int, 3>>* out) {
            for (const hfav_ref& x : d.rules[S->f[f].rule].in) {
                if (S->f[x.field].scalar) continue;
                if (S->f[x.field].inl) expand(x.field, dx + x.off[0], dy + x.off[1], out);
                else out->push_back({x.field, dx + x.off[0], dy + x.off[1]});
            }
        };
    for (int r : p->an.order) {
        if (!in_part(P, r)) continue;
        const int f = d.rules[r].out[0];
        SField& F = S->f[f];
        if (F.inl) continue;
        expand(f, 0, 0, &F.eff);
        int lead = F.eff.empty() ? -1 : -(1 << 20);
        for (auto& e : F.eff) lead = std::max(lead, S->f[e[0]].lead + e[2]);
        F.lead = lead + 1;
    }
    // ring rows: from the oldest row a reader still needs to the newest written,
    // a power of two, so that one unrolled pass of U = max W steps sees every
    // ring at fixed rows
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        if (F.inl || F.scalar || !involved[f]) continue;
        for (int c = 0; c < nf; ++c)
            for (auto& e : S->f[c].eff)
                if (e[0] == f) F.W = std::max(F.W, S->f[c].lead - F.lead - e[2] + 1);
        if (F.load >= 0) F.W = std::max(F.W, 1) + kAhead;
        if (F.W > 0) { int w2 = 1; while (w2 < F.W) w2 *= 2; F.W = w2; }
        S->U = std::max(S->U, F.W);
    }
    S->smem = 0;
    S->ylo = 1 << 20;
    S->yhi = -(1 << 20);
    for (int f = 0; f < nf; ++f) {
        SField& F = S->f[f];
        if (F.inl || !involved[f] || (F.scalar && F.red < 0)) continue;
        if (F.W > 0) {
            F.off = S->smem;
            S->smem += ((size_t)F.W * F.w * es + 15) / 16 * 16;
        }
        S->ylo = std::min(S->ylo, -F.hylo + F.lead);
        S->yhi = std::max(S->yhi, F.hyhi + F.lead);
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
            const bool ring = F.lead - G.lead - e[2] >= 1 && F.lead - G.lead - e[2] + 1 <= G.W - (G.load >= 0 ? kAhead : 0);
            if (!cols || !rows || !ring) return set_error(HFAV_EINVAL, "internal: a rule reads outside its input's ring");
        }
    }
    return HFAV_OK;
}

// each thread takes V columns of a row (tid, tid + NT, ...): the per-step
// work (row checks, fetch set-up, barrier) is shared by V cells.  V = 4 (FP32)
// or 2 (FP64), halved while the rings need more than kSmemDefault of shared
// memory (the default launch limit, less the kernel's static reduction
// buffer); larger rings take an opt-in limit.
constexpr size_t kSmemDefault = 47 * 1024;

int stream_geometry(const hfav_plan_t* p, const Schedule& s, const Part& P, Stream* S) {
    int rc = HFAV_EUNSUPPORTED;
    for (int V = p->dtype == HFAV_F64 ? 2 : 4; V >= 1; V /= 2) {
        *S = Stream();
        rc = stream_geometry_v(p, s, P, V, S);
        if (rc == HFAV_OK && S->smem <= kSmemDefault) return HFAV_OK;
    }
    return rc;
}

// a pointwise part: each CTA row loop loads, computes and stores its cells
// in registers (V columns per thread), no shared memory, no barrier
std::string pointwise_source(const hfav_plan_t* p, const Stream& S, const Part& P, const std::string& name) {
    const Dag& d = p->dag;
    const bool f64 = p->dtype == HFAV_F64;
    const int NT = S.NT, V = S.V, TXc = S.TXc;
    std::ostringstream c;
    c << prelude(f64);
    for (int r : p->an.order)
        if (in_part(P, r)) c << rule_fn(d.rules[r], "hfav_body" + std::to_string(r));
    c << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") " << name << "(";
    // a load may share its array with a goal (in/out): no __restrict__ on loads
    for (size_t a = 0; a < S.loads.size(); ++a) {
        const std::string x = "x" + std::to_string(a), ap = array_params(x, false);
        c << "const T* " << x << ap.substr(ap.find(',')) << ", ";
    }
    for (size_t a = 0; a < S.goals.size(); ++a) c << array_params("y" + std::to_string(a), true) << ", ";
    for (size_t a = 0; a < S.crosses.size(); ++a) c << array_params("z" + std::to_string(a), true) << ", ";
    c << "const double* __restrict__ scal, double* __restrict__ part, int nx, int ny, int CH) {\n"
      << "    const int tid = threadIdx.x, i0 = blockIdx.x * " << TXc << ", j0 = blockIdx.y * CH;\n"
      << "    const int jn = min(CH, ny - j0);\n";
    for (int f : S.scalars) c << "    const T sv" << f << " = (T)scal[" << f << "];\n";
    for (size_t k = 0; k < S.reds.size(); ++k)
        c << red_decl((int)k, d.rules[S.f[S.reds[k]].rule].op == HFAV_OP_REDUCE_MAX, f64);
    c << "    #pragma unroll 1\n"
      << "    for (int r = 0; r < jn; ++r) {\n"
      << "        const int gj = j0 + r;\n";
    for (size_t a = 0; a < S.loads.size(); ++a) {
        const std::string x = "x" + std::to_string(a);
        c << "        const T* const " << x << "r = " << x << " + (long long)(gj + " << x << "_o1) * " << x << "_p1 + " << x
          << "_o0 + i0 + tid;\n";
    }
    for (int kind = 0; kind < 2; ++kind)
        for (size_t a = 0; a < (kind ? S.crosses.size() : S.goals.size()); ++a) {
            const std::string y = (kind ? "z" : "y") + std::to_string(a);
            c << "        T* const " << y << "r = " << y << " + (long long)(gj + " << y << "_o1) * " << y << "_p1 + " << y
              << "_o0 + i0 + tid;\n";
        }
    for (int v = 0; v < V; ++v) {
        c << "        if (i0 + tid + " << v * NT << " < nx) {\n";
        std::function<std::string(int)> read = [&](int g) -> std::string {
            const SField& G = S.f[g];
            if (G.scalar) return "sv" + std::to_string(g);
            if (G.load >= 0) return "x" + std::to_string(G.load) + "r[" + std::to_string(v * NT) + "]";
            const Rule& Q = d.rules[G.rule];
            std::string val = "hfav_body" + std::to_string(G.rule) + "(";
            for (size_t q = 0; q < Q.in.size(); ++q) val += (q ? ", " : "") + read(Q.in[q].field);
            return val + ")";
        };
        for (int r : p->an.order) {
            if (!in_part(P, r)) continue;
            const Rule& R = d.rules[r];
            const int f = R.out[0];
            const SField& F = S.f[f];
            if (F.red >= 0) {
                c << "            { const T in0 = " << read(R.in[0].field) << ";\n"
                  << "              " << red_add(F.red, R.op == HFAV_OP_REDUCE_MAX, f64, "in0") << " }\n";
                continue;
            }
            if (F.goal < 0 && F.cross < 0) continue;   // inlined into its readers
            c << "            { const T v = hfav_body" << r << "(";
            for (size_t q = 0; q < R.in.size(); ++q) c << (q ? ", " : "") << read(R.in[q].field);
            c << ");\n";
            if (F.goal >= 0) c << "              y" << F.goal << "r[" << v * NT << "] = v;\n";
            if (F.cross >= 0) c << "              z" << F.cross << "r[" << v * NT << "] = v;\n";
            c << "            }\n";
        }
        c << "        }\n";
    }
    c << "    }\n";
    if (!S.reds.empty()) {
        c << "    __shared__ double hfav_red[" << NT / 32 << "];\n"
          << "    const long long cta = (long long)blockIdx.y * gridDim.x + blockIdx.x, nb = (long long)gridDim.x * gridDim.y;\n";
        for (size_t k = 0; k < S.reds.size(); ++k) {
            const bool mx = d.rules[S.f[S.reds[k]].rule].op == HFAV_OP_REDUCE_MAX;
            const std::string op = mx ? "fmax(a, b)" : "a + b";
            c << "    {\n"
              << "        double a = " << red_final((int)k, mx, f64) << ";\n"
              << "        for (int o = 16; o > 0; o >>= 1) { const double b = __shfl_xor_sync(0xffffffffu, a, o); a = " << op
              << "; }\n"
              << "        __syncthreads();\n"
              << "        if ((tid & 31) == 0) hfav_red[tid >> 5] = a;\n"
              << "        __syncthreads();\n"
              << "        if (tid == 0) {\n"
              << "            for (int w = 1; w < " << NT / 32 << "; ++w) { const double b = hfav_red[w]; a = " << op << "; }\n"
              << "            part[" << k << " * nb + cta] = a;\n"
              << "        }\n"
              << "    }\n";
        }
    }
    c << "}\n";
    return c.str();
}

std::string stream_source(const hfav_plan_t* p, const Stream& S, const Part& P, const std::string& name) {
    if (S.pointwise) return pointwise_source(p, S, P, name);
    const Dag& d = p->dag;
    const bool f64 = p->dtype == HFAV_F64;
    const int NT = S.NT, TXc = S.TXc, V = S.V;
    auto slot = [](const std::string& row, int W) {   // ring row of a (possibly negative) row index
        return "((unsigned)(" + row + " + " + std::to_string(1024 * W) + ") % " + std::to_string(W) + "u)";
    };
    // a thread's columns tid + v NT, v < V, of a ring row of width w: the
    // condition that column set v is inside ("" when always, "-" never)
    auto inside = [&](int v, int w) -> std::string {
        if (w - v * NT >= NT) return "";
        if (w - v * NT <= 0) return "-";
        return "tid < " + std::to_string(w - v * NT);
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
    for (int r : p->an.order)
        if (in_part(P, r)) c << rule_fn(d.rules[r], "hfav_body" + std::to_string(r));
    c << "extern \"C\" __global__ void __launch_bounds__(" << NT << ") " << name << "(";
    // an in-place load shares its array with a goal: no __restrict__ on it
    for (size_t a = 0; a < S.loads.size(); ++a)
        c << (S.inplace[a] ? "const T* " + ("x" + std::to_string(a)) + array_params("x" + std::to_string(a), false).substr(
                                 array_params("x" + std::to_string(a), false).find(','))
                           : array_params("x" + std::to_string(a), false))
          << ", ";
    for (size_t a = 0; a < S.goals.size(); ++a) c << array_params("y" + std::to_string(a), true) << ", ";
    for (size_t a = 0; a < S.crosses.size(); ++a) c << array_params("z" + std::to_string(a), true) << ", ";
    for (size_t a = 0; a < S.loads.size(); ++a)
        if (S.inplace[a]) c << "const T* __restrict__ cb" << a << ", const T* __restrict__ rb" << a << ", ";
    c << "const double* __restrict__ scal, double* __restrict__ part, int nx, int ny, int CH) {\n"
      << "    extern __shared__ __align__(16) unsigned char smem[];\n"
      << "    const int tid = threadIdx.x, i0 = blockIdx.x * " << TXc << ", j0 = blockIdx.y * CH;\n"
      << "    const int jn = min(CH, ny - j0);\n"
      << "    const bool last_x = i0 + " << TXc << " >= nx, last_y = j0 + jn >= ny;\n";
    for (int f = 0; f < d.n_fields; ++f)
        if (!S.f[f].inl && S.f[f].W > 0) c << "    T* s" << f << " = (T*)(smem + " << S.f[f].off << ");\n";
    for (int f : S.scalars) c << "    const T sv" << f << " = (T)scal[" << f << "];\n";
    for (size_t k = 0; k < S.reds.size(); ++k)
        c << red_decl((int)k, d.rules[S.f[S.reds[k]].rule].op == HFAV_OP_REDUCE_MAX, f64);
    // fields read from memory: each thread's columns (fixed), a row fetch
    // issued kAhead steps ahead, indices wrapped (periodic axioms) or clamped
    // into the field's footprint.  A field whose array the part also writes
    // (a declared in/out pair) reads only its own strip's interior rows live:
    // the halo columns and the rows beyond its chunk come from bands saved
    // before the launch, since neighbouring CTAs overwrite them.
    const bool any_inplace = std::find(S.inplace.begin(), S.inplace.end(), 1) != S.inplace.end();
    if (any_inplace) c << "    const int wint = min(" << TXc << ", nx - i0);\n";
    for (int f : S.loads) {
        const SField& F = S.f[f];
        const std::string a = std::to_string(F.load), x = "x" + a;
        const bool inpl = S.inplace[F.load];
        const int HXa = std::max(1, F.hxlo + F.hxhi), HYa = std::max(1, F.hylo + F.hyhi);
        for (int v = 0; v < V; ++v) {
            const std::string cv = a + "_" + std::to_string(v);
            if (inside(v, F.w) == "-") continue;
            if (!inpl) {
                c << "    int col" << cv << " = i0 - " << F.hxlo << " + tid + " << v * NT << ";\n"
                  << "    if (" << x << "_w) col" << cv << " = hfav_wrap(col" << cv << ", nx);\n"
                  << "    else col" << cv << " = min(max(col" << cv << ", -" << F.hxlo << "), nx - 1 + " << F.hxhi << ");\n"
                  << "    const T* src" << cv << " = " << x << " + col" << cv << " + " << x << "_o0;\n";
            } else {
                c << "    const int xv" << cv << " = tid + " << v * NT - F.hxlo << ";\n"
                  << "    const bool live" << cv << " = xv" << cv << " >= 0 && xv" << cv << " < wint;\n"
                  << "    const int kb" << cv << " = min(max(xv" << cv << " < 0 ? xv" << cv << " + " << F.hxlo << " : "
                  << F.hxlo << " + xv" << cv << " - wint, 0), " << HXa - 1 << ");\n"
                  << "    const T* src" << cv << " = live" << cv << " ? " << x << " + (long long)" << x << "_o1 * " << x
                  << "_p1 + " << x << "_o0 + i0 + xv" << cv << " : cb" << a << " + ((long long)blockIdx.x * (ny + "
                  << F.hylo + F.hyhi << ") + " << F.hylo << ") * " << HXa << " + kb" << cv << ";\n"
                  << "    const long long sr" << cv << " = live" << cv << " ? " << x << "_p1 : " << HXa << ";\n"
                  << "    const T* pl" << cv << " = src" << cv << " + (long long)(j0 + " << S.ylo << ") * sr" << cv << ";\n"
                  << "    const int rcol" << cv << " = min(max(i0 + xv" << cv << " + " << F.hxlo << ", 0), nx + "
                  << F.hxlo + F.hxhi - 1 << ");\n";
            }
        }
        c << "    auto fetch" << a << " = [&](int r) {\n"
          << "        if (r >= -" << F.hylo << " && r < jn + " << F.hyhi << ") {\n";
        if (!inpl) {
            c << "            int gj = j0 + r;\n"
              << "            if (" << x << "_w) gj = hfav_wrap(gj, ny);\n"
              << "            else gj = min(max(gj, -" << F.hylo << "), ny - 1 + " << F.hyhi << ");\n"
              << "            const long long ro = (long long)(gj + " << x << "_o1) * " << x << "_p1;\n";
        } else {
            c << "            const bool band = r < 0 || r >= jn;\n"
              << "            const T* const rrow = rb" << a << " + ((long long)blockIdx.y * " << HYa << " + min(max(r < 0 ? r + "
              << F.hylo << " : " << F.hylo << " + r - jn, 0), " << HYa - 1 << ")) * (nx + " << F.hxlo + F.hxhi << ");\n";
        }
        c << "            T* const dst = s" << f << " + " << slot("r", F.W) << " * " << F.w << " + tid;\n";
        for (int v = 0; v < V; ++v) {
            const std::string in = inside(v, F.w), cv = a + "_" + std::to_string(v);
            if (in == "-") continue;
            c << "            " << (in.empty() ? "" : "if (" + in + ") ") << "hfav_cp(dst + " << v * NT << ", ";
            if (!inpl) c << "src" << cv << " + ro);\n";
            else c << "band ? rrow + rcol" << cv << " : pl" << cv << ");\n";
        }
        c << "        }\n";
        // the fetches run for consecutive rows: each thread's live row pointers step by one row
        if (inpl)
            for (int v = 0; v < V; ++v)
                if (inside(v, F.w) != "-") c << "        pl" << a << "_" << v << " += sr" << a << "_" << v << ";\n";
        c << "    };\n";
    }
    // written fields: each thread's column pointers (fixed); caller goals take
    // the interior, crossing arrays the cells of their footprint this CTA owns
    // (the interior part of its strip and chunk, plus the outer halo at the
    // grid's edges)
    for (int f = 0; f < d.n_fields; ++f) {
        const SField& F = S.f[f];
        for (int kind = 0; kind < 2; ++kind) {
            const int idx = kind == 0 ? F.goal : F.cross;
            if (idx < 0) continue;
            const std::string y = (kind == 0 ? "y" : "z") + std::to_string(idx);
            for (int v = 0; v < V; ++v) {
                const std::string g = y + "_" + std::to_string(v);
                if (inside(v, F.w) == "-") continue;
                c << "    const int gx" << g << " = tid + " << v * NT - F.hxlo << ";\n";
                if (kind == 0)
                    c << "    const bool gok" << g << " = gx" << g << " >= 0 && gx" << g << " < " << TXc << " && i0 + gx" << g
                      << " < nx;\n";
                else
                    c << "    const bool gok" << g << " = (gx" << g << " >= 0 && gx" << g << " < " << TXc << " && i0 + gx"
                      << g << " < nx) || (i0 + gx" << g << " < 0) || (last_x && i0 + gx" << g << " >= nx && i0 + gx" << g
                      << " < nx + " << F.hxhi << ");\n";
                c << "    T* const gcol" << g << " = " << y << " + (long long)" << y << "_o1 * " << y << "_p1 + (i0 + gx" << g
                  << " + " << y << "_o0);\n";
            }
        }
    }
    c << "    #pragma unroll 1\n"
      << "    for (int r = " << S.ylo << "; r < " << S.ylo + kAhead << "; ++r) {\n";
    for (int f : S.loads) c << "        fetch" << S.f[f].load << "(r);\n";
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
        for (int f : S.loads) c << "        fetch" << S.f[f].load << "(s + " << kAhead << ");\n";
        c << "        hfav_commit();\n";
        for (int r : p->an.order) {
            if (!in_part(P, r)) continue;
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
                    if (G.scalar) return "sv" + std::to_string(g);
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
                if (F.red >= 0) {
                    // a reduction: the input's value over this CTA's interior cells
                    const std::string x = "(tid + " + std::to_string(v * NT - F.hxlo) + ")";
                    c << "                if (" << x << " < " << TXc << " && i0 + " << x << " < nx)\n"
                      << "                    " << red_add(F.red, R.op == HFAV_OP_REDUCE_MAX, f64, "in0") << "\n";
                    c << "            }\n";
                    continue;
                }
                c << "                const T v = " << rule_call(R, "hfav_body" + std::to_string(r)) << ";\n";
                if (F.W > 0)
                    c << "                s" << f << "[" << cslot(k, F.lead, 0, F.W) * F.w + v * NT << " + tid] = v;\n";
                if (F.goal >= 0) {
                    const std::string g = "y" + std::to_string(F.goal) + "_" + std::to_string(v);
                    c << "                if (r >= 0 && r < jn && gok" << g << ")\n"
                      << "                    gcol" << g << "[(long long)(j0 + r) * y" << F.goal << "_p1] = v;\n";
                }
                if (F.cross >= 0) {
                    const std::string g = "z" + std::to_string(F.cross) + "_" + std::to_string(v);
                    c << "                if (gok" << g << " && ((r >= 0 && r < jn) || j0 + r < 0 || (last_y && j0 + r >= ny)))\n"
                      << "                    gcol" << g << "[(long long)(j0 + r) * z" << F.cross << "_p1] = v;\n";
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
      << "    asm volatile(\"cp.async.wait_all;\\n\" ::: \"memory\");\n";
    // one partial per CTA and reduction, combined in a fixed order
    if (!S.reds.empty()) {
        c << "    __shared__ double hfav_red[" << NT / 32 << "];\n"
          << "    const long long cta = (long long)blockIdx.y * gridDim.x + blockIdx.x, nb = (long long)gridDim.x * gridDim.y;\n";
        for (size_t k = 0; k < S.reds.size(); ++k) {
            const bool mx = d.rules[S.f[S.reds[k]].rule].op == HFAV_OP_REDUCE_MAX;
            const std::string op = mx ? "fmax(a, b)" : "a + b";
            c << "    {\n"
              << "        double a = " << red_final((int)k, mx, f64) << ";\n"
              << "        for (int o = 16; o > 0; o >>= 1) { const double b = __shfl_xor_sync(0xffffffffu, a, o); a = " << op
              << "; }\n"
              << "        __syncthreads();\n"
              << "        if ((tid & 31) == 0) hfav_red[tid >> 5] = a;\n"
              << "        __syncthreads();\n"
              << "        if (tid == 0) {\n"
              << "            for (int w = 1; w < " << NT / 32 << "; ++w) { const double b = hfav_red[w]; a = " << op << "; }\n"
              << "            part[" << k << " * nb + cta] = a;\n"
              << "        }\n"
              << "    }\n";
        }
    }
    c << "}\n";
    return c.str();
}

// the finalization after a part with reductions: one CTA combines each
// reduction's partials in a fixed order (so runs are bitwise repeatable), then
// evaluates, in FP64, the scalar rules whose inputs are now known
std::string finalize_source(const hfav_plan_t* p, const std::vector<int>& red_fields, const std::vector<int>& rules) {
    const Dag& d = p->dag;
    std::ostringstream c;
    c << prelude(true);
    for (int r : rules) c << rule_fn(d.rules[r], "hfav_body" + std::to_string(r));
    c << "extern \"C\" __global__ void __launch_bounds__(256) hfav_cg_finalize(const double* __restrict__ part, "
      << "long long nparts, double* __restrict__ scal) {\n"
      << "    __shared__ double red[8];\n"
      << "    const int tid = threadIdx.x;\n";
    for (size_t k = 0; k < red_fields.size(); ++k) {
        const int f = red_fields[k];
        int rr = -1;
        for (size_t r = 0; r < d.rules.size(); ++r) if (d.rules[r].out[0] == f) rr = (int)r;
        const bool mx = d.rules[rr].op == HFAV_OP_REDUCE_MAX;
        const std::string op = mx ? "fmax(a, b)" : "a + b";
        c << "    {\n"
          << "        double a = " << (mx ? "__longlong_as_double(0xfff0000000000000ULL)" : "0.0") << ";\n"
          << "        for (long long i = tid; i < nparts; i += 256) { const double b = part[" << k << " * nparts + i]; a = "
          << op << "; }\n"
          << "        for (int o = 16; o > 0; o >>= 1) { const double b = __shfl_xor_sync(0xffffffffu, a, o); a = " << op
          << "; }\n"
          << "        if ((tid & 31) == 0) red[tid >> 5] = a;\n"
          << "        __syncthreads();\n"
          << "        if (tid == 0) {\n"
          << "            for (int w = 1; w < 8; ++w) { const double b = red[w]; a = " << op << "; }\n"
          << "            scal[" << f << "] = a;\n"
          << "        }\n"
          << "        __syncthreads();\n"
          << "    }\n";
    }
    if (!rules.empty()) {
        c << "    if (tid == 0) {\n";
        for (int r : rules) {
            const Rule& R = d.rules[r];
            c << "        scal[" << R.out[0] << "] = hfav_body" << r << "(";
            for (size_t k = 0; k < R.in.size(); ++k) c << (k ? ", " : "") << "scal[" << R.in[k].field << "]";
            c << ");\n";
        }
        c << "    }\n";
    }
    c << "}\n";
    return c.str();
}

// The parts of a plan in execution order: the analysis's fusion groups
// (fused) or single rules (unfused), scalar rules set aside for the
// finalizations.  Also: after each part, the scalar rules it makes ready.
struct Program {
    std::vector<Part> parts;
    std::vector<std::vector<int>> fin_reds;    // per part: rank-0 fields its reductions write
    std::vector<std::vector<int>> fin_rules;   // per part: scalar rules evaluated after it
};

int make_program(const hfav_plan_t* p, bool fused, Program* G) {
    const Dag& d = p->dag;
    const int nr = (int)d.rules.size();
    auto scalar_rule = [&](int r) {
        for (const hfav_ref& x : d.rules[r].in) if (d.rank[x.field] != 0) return false;
        return d.rank[d.rules[r].out[0]] == 0;
    };
    std::map<int, int> part_of_group;
    std::vector<int> part_of(nr, -1);
    std::vector<Part> parts;
    for (int r : p->an.order) {
        if (scalar_rule(r)) continue;
        int k;
        if (fused) {
            auto it = part_of_group.find(p->an.rule_group[r]);
            if (it == part_of_group.end()) {
                k = (int)parts.size();
                part_of_group[p->an.rule_group[r]] = k;
                parts.push_back(Part());
            } else {
                k = it->second;
            }
        } else {
            k = (int)parts.size();
            parts.push_back(Part());
        }
        parts[k].rules.push_back(r);
        part_of[r] = k;
    }
    // execution order: a part runs after every part whose grid fields or
    // scalars it reads
    std::vector<int> producer(d.n_fields, -1);
    for (int r = 0; r < nr; ++r) producer[d.rules[r].out[0]] = r;
    std::function<void(int, std::set<int>*)> sources = [&](int f, std::set<int>* out) {
        const int r = producer[f];
        if (r < 0) return;
        if (part_of[r] >= 0) { out->insert(part_of[r]); return; }
        for (const hfav_ref& x : d.rules[r].in) sources(x.field, out);   // a scalar rule: its inputs' parts
    };
    const int np = (int)parts.size();
    std::vector<std::set<int>> deps(np);
    for (int k = 0; k < np; ++k)
        for (int r : parts[k].rules)
            for (const hfav_ref& x : d.rules[r].in) {
                std::set<int> src;
                sources(x.field, &src);
                for (int q : src) if (q != k) deps[k].insert(q);
            }
    std::vector<char> done(np, 0);
    std::vector<char> scal_ready(d.n_fields, 0), scal_done(nr, 0);
    for (int step = 0; step < np; ++step) {
        int pick = -1;
        for (int k = 0; k < np && pick < 0; ++k) {
            if (done[k]) continue;
            bool ok = true;
            for (int q : deps[k]) if (!done[q]) ok = false;
            if (ok) pick = k;
        }
        if (pick < 0) return set_error(HFAV_EUNSUPPORTED, "the DAG's parts form a cycle");
        done[pick] = 1;
        G->parts.push_back(parts[pick]);
        std::vector<int> reds, rules;
        for (int r : parts[pick].rules)
            if (d.rank[d.rules[r].out[0]] == 0) { reds.push_back(d.rules[r].out[0]); scal_ready[d.rules[r].out[0]] = 1; }
        for (bool more = true; more;) {
            more = false;
            for (int r : p->an.order) {
                if (!scalar_rule(r) || scal_done[r]) continue;
                bool ok = true;
                for (const hfav_ref& x : d.rules[r].in) if (!scal_ready[x.field]) ok = false;
                if (!ok) continue;
                scal_done[r] = 1;
                scal_ready[d.rules[r].out[0]] = 1;
                rules.push_back(r);
                more = true;
            }
        }
        G->fin_reds.push_back(reds);
        G->fin_rules.push_back(rules);
    }
    return HFAV_OK;
}

bool has_scalars(const hfav_plan_t* p) {
    for (int rk : p->dag.rank) if (rk == 0) return true;
    return false;
}

// the loads of a single-part program whose arrays a declared in/out goal shares
void mark_inplace(const hfav_plan_t* p, Stream* S, void* const* ax, void* const* go) {
    const Dag& d = p->dag;
    for (size_t l = 0; l < S->loads.size(); ++l)
        for (size_t k = 0; k < d.goals.size(); ++k) {
            const int a = d.inout[k];
            if (a >= 0 && d.axioms[a] == S->loads[l] && (!ax || go[k] == ax[a])) S->inplace[l] = 1;
        }
}

// ---- fused 2D, placement reg: warp strips ------------------------------------------
// Each warp owns a strip of 32 V columns (V consecutive cells per lane) and a
// chunk of R rows, and streams down the chunk.  Every field the part loads or
// stores keeps a window of its last rows in registers (Sec. 3.5
// "Contraction", with the rolling buffer in the register file), the
// i-neighbours cross lanes by warp shuffle (offsets up to V cells), and the
// strips overlap by the part's footprint in x, so no lane needs data from
// beyond its strip: no shared memory and no barrier.  A field computed at
// step t holds row t - Y0 - lead (its lead puts every row it reads at or
// before its inputs' current rows, so one pass over the fields in
// topological order per step suffices); loads arrive P rows ahead.  Windows
// are powers of two and the step loop is unrolled by the largest, so every
// window slot is a constant of the unrolled code.  Taken for one-part DAGs
// without reductions whose reads reach at most V cells across; a run whose
// goal shares its array with an input (declared in/out) takes the ring
// kernel instead.
struct WStrip {
    int V = 1, NT = 0, HL = 0, TXw = 0, M = 1, P = 3, Y0 = 0, fill = 0;   // P: rows a load runs ahead (at least 3)
    std::vector<int> lead, NW, order;   // per field; order: stored fields computed here, topological
};

int wstrip_geometry(const hfav_plan_t* p, const Schedule& s, const Part& P, const Stream& S, WStrip* G) {
    const Dag& d = p->dag;
    const int nf = d.n_fields;
    if (S.pointwise || !S.reds.empty() || !S.crosses.empty() || !S.scalars.empty())
        return set_error(HFAV_EUNSUPPORTED, "warp strips take one-part DAGs without reductions or scalars");
    const int V = p->dtype == HFAV_F64 ? 2 : 4;
    G->V = V;
    G->NT = s.tx * s.ty;
    int HL = 0, HR = 0;
    for (int f = 0; f < nf; ++f)
        if (!S.f[f].scalar && (S.f[f].rule >= 0 || S.f[f].load >= 0)) {
            HL = std::max(HL, S.f[f].hxlo);
            HR = std::max(HR, S.f[f].hxhi);
        }
    G->HL = (HL + V - 1) / V * V;
    G->TXw = (32 * V - G->HL - HR) / V * V;
    if (G->TXw < 16 * V) return set_error(HFAV_EUNSUPPORTED, "this DAG's footprint is too wide for warp strips");
    G->lead.assign(nf, 0);
    G->NW.assign(nf, 0);
    G->order.clear();
    for (int r : p->an.order) {
        if (!in_part(P, r)) continue;
        const int f = d.rules[r].out[0];
        if (S.f[f].inl) continue;
        int lead = -(1 << 20);
        for (auto& e : S.f[f].eff) {
            if (e[1] > V || e[1] < -V) return set_error(HFAV_EUNSUPPORTED, "warp strips take reads within V cells in x");
            lead = std::max(lead, G->lead[e[0]] + e[2]);
        }
        if (S.f[f].eff.empty()) lead = 0;
        G->lead[f] = lead;
        G->order.push_back(f);
    }
    // window rows: from the newest row of a field to the oldest a reader takes
    size_t regs = 0;
    G->M = 1;
    G->Y0 = 0;
    for (int f : S.loads) G->Y0 = std::max(G->Y0, S.f[f].hylo);
    int fill = 0;
    std::vector<int> span(nf, 1);
    int P_max = 1 << 20;
    for (int f = 0; f < nf; ++f) {
        const SField& F = S.f[f];
        if (F.scalar || (F.rule < 0 && F.load < 0) || F.inl) continue;
        int w = 1;
        for (int c : G->order)
            for (auto& e : S.f[c].eff)
                if (e[0] == f) w = std::max(w, G->lead[c] - G->lead[f] - e[2] + 1);
        span[f] = w;
        if (F.load >= 0) w += G->P;
        int w2 = 1;
        while (w2 < w) w2 *= 2;
        G->NW[f] = w2;
        if (F.load >= 0) P_max = std::min(P_max, w2 - span[f]);
        G->M = std::max(G->M, w2);
        regs += (size_t)w2 * V * (p->dtype == HFAV_F64 ? 2 : 1);
        fill = std::max(fill, F.hyhi + G->lead[f]);
    }
    // loads run as far ahead as their (power-of-two) windows leave room for
    if (!S.loads.empty()) G->P = P_max;
    if (regs > 160) return set_error(HFAV_EUNSUPPORTED, "this DAG's row windows exceed the register budget of warp strips");
    G->fill = G->Y0 + fill;
    return HFAV_OK;
}

// positive remainder of a (possibly negative) row index
int pmod(int a, int n) { return ((a % n) + n) % n; }

std::string wstrip_source(const hfav_plan_t* p, const Stream& S, const Part& P, const WStrip& G, const std::string& name) {
    const Dag& d = p->dag;
    const bool f64 = p->dtype == HFAV_F64;
    const int V = G.V, M = G.M;
    const std::string VT = f64 ? "double2" : (V == 4 ? "float4" : "float2");
    const int VB = V * (f64 ? 8 : 4);   // bytes of a lane's cells in one row
    const char* comp[4] = {"x", "y", "z", "w"};
    // window slot sl of field f: one vector of a lane's V cells of one row,
    // so a load lands in it with no copy and a goal row leaves from it
    auto wv = [](int f, int slot) { return "w" + std::to_string(f) + "_" + std::to_string(slot); };
    auto we = [&](int f, int slot, int e) { return wv(f, slot) + "." + comp[e]; };
    std::ostringstream c;
    c << prelude(f64);
    for (int r : p->an.order)
        if (in_part(P, r)) c << rule_fn(d.rules[r], "hfav_body" + std::to_string(r));
    c << "extern \"C\" __global__ void __launch_bounds__(" << G.NT << ") " << name << "(";
    for (size_t a = 0; a < S.loads.size(); ++a) c << array_params("x" + std::to_string(a), false) << ", ";
    for (size_t a = 0; a < S.goals.size(); ++a) c << array_params("y" + std::to_string(a), true) << ", ";
    c << "int nx, int ny, int R, int nstrips, int sh) {\n"
      << "    const int lane = threadIdx.x & 31;\n"
      << "    const long long wid = ((long long)blockIdx.x * " << G.NT << " + threadIdx.x) >> 5;\n"
      << "    const int strip = (int)(wid % nstrips), j0 = (int)(wid / nstrips) * R;\n"
      << "    if (j0 >= ny) return;   // the whole warp\n"
      << "    const int Rr = min(R, ny - j0), nstep = Rr + " << G.fill << ";\n"
      << "    const int s0 = strip * " << G.TXw << " - " << G.HL << " - sh, c0 = s0 + " << V << " * lane;\n"
      << "    const int lo = max(s0 + " << G.HL << ", 0), hi = min(s0 + " << G.HL + G.TXw << ", nx);\n";
    // loads: fixed columns per lane (wrapped or clamped into the footprint);
    // a warp whose lanes' cells all lie contiguous and 16-byte aligned in
    // every load takes the vector loop
    std::string vall = "true";
    for (int f : S.loads) {
        const SField& F = S.f[f];
        const std::string a = std::to_string(F.load), x = "x" + a;
        for (int e = 0; e < V; ++e)
            c << "    int cx" << a << "_" << e << " = c0 + " << e << ";\n"
              << "    cx" << a << "_" << e << " = " << x << "_w ? hfav_wrap(cx" << a << "_" << e << ", nx) : min(max(cx" << a
              << "_" << e << ", -" << F.hxlo << "), nx - 1 + " << F.hxhi << ");\n";
        c << "    const bool vx" << a << " = c0 >= 0 && c0 + " << V << " <= nx && ((" << x << "_o0 + c0) & " << V - 1
          << ") == 0 && (" << x << "_p1 & " << V - 1 << ") == 0 && ((unsigned long long)" << x << " & " << VB - 1
          << ") == 0;\n";
        vall += " && vx" + a;
    }
    for (size_t q = 0; q < S.goals.size(); ++q) {
        const std::string y = "y" + std::to_string(q);
        c << "    const bool vy" << q << " = c0 >= lo && c0 + " << V << " <= hi && ((" << y << "_o0 + c0) & " << V - 1
          << ") == 0 && (" << y << "_p1 & " << V - 1 << ") == 0 && ((unsigned long long)" << y << " & " << VB - 1
          << ") == 0;\n";
    }
    for (int f = 0; f < d.n_fields; ++f)
        for (int sl = 0; sl < G.NW[f]; ++sl) c << "    " << VT << " " << wv(f, sl) << " = {};\n";
    // a load of row `row` (an expression; rows past the footprint are
    // wrapped or clamped like any other, so every load is unconditional)
    auto emit_load = [&](std::ostringstream& o, int f, const std::string& row, int sl, bool vec, const std::string& ind) {
        const SField& F = S.f[f];
        const std::string a = std::to_string(F.load), x = "x" + a;
        o << ind << "{\n"
          << ind << "    int gj = j0 + " << row << ";\n"
          << ind << "    gj = " << x << "_w ? hfav_wrap(gj, ny) : min(max(gj, -" << F.hylo << "), ny - 1 + " << F.hyhi
          << ");\n"
          << ind << "    const T* rp = " << x << " + (long long)(gj + " << x << "_o1) * " << x << "_p1 + " << x << "_o0;\n";
        // the loads are volatile asm, so the compiler keeps them where they
        // are issued (rows ahead of their readers) instead of sinking them
        // into the later step that reads them
        if (vec) {
            o << ind << "    asm volatile(\"ld.global.nc.v" << V << "." << (f64 ? "f64" : "f32") << " {";
            for (int e = 0; e < V; ++e) o << (e ? ", " : "") << "%" << e;
            o << "}, [%" << V << "];\" : ";
            for (int e = 0; e < V; ++e) o << (e ? ", " : "") << "\"=" << (f64 ? "d" : "f") << "\"(" << we(f, sl, e) << ")";
            o << " : \"l\"(rp + c0));\n";
        } else {
            for (int e = 0; e < V; ++e)
                o << ind << "    asm volatile(\"ld.global.nc." << (f64 ? "f64" : "f32") << " %0, [%1];\" : \"="
                  << (f64 ? "d" : "f") << "\"(" << we(f, sl, e) << ") : \"l\"(rp + cx" << a << "_" << e << "));\n";
        }
        o << ind << "}\n";
    };
    auto emit_main = [&](std::ostringstream& o, bool vec) {
        for (int f : S.loads)
            for (int q = 0; q < G.P; ++q) emit_load(o, f, std::to_string(q - G.Y0), pmod(q - G.Y0, G.NW[f]), vec, "        ");
        o << "        #pragma unroll 1\n"
          << "        for (int t0 = 0; t0 < nstep; t0 += " << M << ") {\n";
        for (int k = 0; k < M; ++k) {
            o << "        if (t0 + " << k << " < nstep) {   // step t0 + " << k << "\n"
              << "            const int t = t0 + " << k << ";\n";
            for (int f : S.loads)
                emit_load(o, f, "t + " + std::to_string(G.P - G.Y0), pmod(k + G.P - G.Y0, G.NW[f]), vec, "            ");
            for (int f : G.order) {
                const SField& F = S.f[f];
                const Rule& R = d.rules[F.rule];
                const int lf = G.lead[f];
                // the value of field g, shifted by (dx, dy), at cell e of this
                // lane; each shuffle is declared once per step
                std::set<std::string> shuf;
                std::ostringstream sh;
                std::function<std::string(int, int, int, int)> read = [&](int g, int e, int dx, int dy) -> std::string {
                    const SField& Gf = S.f[g];
                    if (Gf.inl) {
                        const Rule& Q = d.rules[Gf.rule];
                        std::string val = "hfav_body" + std::to_string(Gf.rule) + "(";
                        for (size_t q = 0; q < Q.in.size(); ++q)
                            val += (q ? ", " : "") + read(Q.in[q].field, e, dx + Q.in[q].off[0], dy + Q.in[q].off[1]);
                        return val + ")";
                    }
                    const int sl = pmod(k - G.Y0 - lf + dy, G.NW[g]);
                    const int ee = e + dx;
                    if (ee >= 0 && ee < V) return we(g, sl, ee);
                    const bool left = ee < 0;
                    const int src = left ? ee + V : ee - V;
                    const std::string nm = std::string(left ? "sl" : "sr") + std::to_string(g) + "_" + std::to_string(sl) +
                                           "_" + std::to_string(src);
                    if (shuf.insert(nm).second)
                        sh << "                const T " << nm << " = " << (left ? "__shfl_up_sync" : "__shfl_down_sync")
                           << "(0xffffffffu, " << we(g, sl, src) << ", 1);\n";
                    return nm;
                };
                std::ostringstream body;
                const int sl_f = pmod(k - G.Y0 - lf, G.NW[f]);
                for (int e = 0; e < V; ++e) {
                    body << "                {\n";
                    for (size_t q = 0; q < R.in.size(); ++q)
                        body << "                    const T in" << q << " = "
                             << read(R.in[q].field, e, R.in[q].off[0], R.in[q].off[1]) << ";\n";
                    body << "                    " << we(f, sl_f, e) << " = "
                         << rule_call(R, "hfav_body" + std::to_string(F.rule)) << ";\n"
                         << "                }\n";
                }
                o << "            {\n"
                  << "                const int row = t - " << G.Y0 + lf << ";\n"
                  << "                if (row >= -" << F.hylo << " && row < Rr + " << F.hyhi << ") {\n"
                  << sh.str() << body.str();
                if (F.goal >= 0) {
                    const std::string y = "y" + std::to_string(F.goal);
                    o << "                if (row >= 0 && row < Rr) {\n"
                      << "                    T* const yr = " << y << " + (long long)(j0 + row + " << y << "_o1) * " << y
                      << "_p1 + " << y << "_o0;\n"
                      << "                    if (vy" << F.goal << ") {\n"
                      << "                        *(" << VT << "*)(yr + c0) = " << wv(f, sl_f) << ";\n"
                      << "                    } else {\n";
                    for (int e = 0; e < V; ++e)
                        o << "                        if (c0 + " << e << " >= lo && c0 + " << e << " < hi) yr[c0 + " << e
                          << "] = " << we(f, sl_f, e) << ";\n";
                    o << "                    }\n"
                      << "                }\n";
                }
                o << "                }\n"
                  << "            }\n";
            }
            o << "        }\n";
        }
        o << "        }\n";
    };
    std::ostringstream mv, ms;
    emit_main(mv, true);
    emit_main(ms, false);
    c << "    if (__all_sync(0xffffffffu, " << vall << ")) {\n" << mv.str() << "    } else {\n" << ms.str() << "    }\n"
      << "}\n";
    return c.str();
}

}  // namespace

bool codegen_inplace(const hfav_plan_t* p, const Schedule& s) {
    if (p->pipeline != PIPE_CODEGEN || s.fusion == FUSE_UNFUSED || p->dag.ndim != 2) return false;
    Program G;
    if (make_program(p, true, &G)) return false;
    return G.parts.size() == 1;
}

bool codegen_wstrip_ok(const hfav_plan_t* p, const Schedule& s, std::string* why) {
    Program G;
    Stream S;
    WStrip W;
    int rc = make_program(p, true, &G);
    if (!rc && G.parts.size() != 1) rc = set_error(HFAV_EUNSUPPORTED, "warp strips take one-part DAGs");
    if (!rc) rc = stream_geometry(p, s, G.parts[0], &S);
    if (!rc) rc = wstrip_geometry(p, s, G.parts[0], S, &W);
    if (rc && why) *why = std::string("full:reg for generated kernels: ") + hfav_last_error();
    return rc == HFAV_OK;
}

int plan_source(const hfav_plan_t* p, std::string* out) {
    if (p->pipeline != PIPE_CODEGEN) return set_error(HFAV_EUNSUPPORTED, "the plan runs no generated kernels");
    std::ostringstream o;
    if (p->sched.fusion != FUSE_UNFUSED || has_scalars(p)) {
        Program G;
        int rc = make_program(p, p->sched.fusion != FUSE_UNFUSED, &G);
        if (rc) return rc;
        const bool inpl = codegen_inplace(p, p->sched);
        for (size_t k = 0; k < G.parts.size(); ++k) {
            Stream S;
            if ((rc = stream_geometry(p, p->sched, G.parts[k], &S))) return rc;
            if (p->sched.placement == PLACE_REG) {   // warp strips (a run whose goal aliases an input takes the ring kernel)
                WStrip W;
                if ((rc = wstrip_geometry(p, p->sched, G.parts[k], S, &W))) return rc;
                o << "// ---- kernel " << k << "\n" << wstrip_source(p, S, G.parts[k], W, "hfav_cg_wstrip");
                continue;
            }
            if (inpl) mark_inplace(p, &S, nullptr, nullptr);   // the declared pairs, as an aliased run compiles them
            o << "// ---- kernel " << k << "\n" << stream_source(p, S, G.parts[k], "hfav_cg_part");
            if (!G.fin_reds[k].empty() || !G.fin_rules[k].empty())
                o << "// ---- kernel " << k << " finalize\n" << finalize_source(p, G.fin_reds[k], G.fin_rules[k]);
        }
        *out = o.str();
        return HFAV_OK;
    }
    for (int r : p->an.order) {
        const Rule& R = p->dag.rules[r];
        if (R.op != HFAV_OP_EXPR) continue;
        std::vector<int> fields;
        const std::vector<int> slot = rule_slots(R, &fields);
        o << "// ---- kernel rule " << r << "\n" << rule_source(p, R, slot, (int)fields.size());
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
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)device_sms() * 16));
    HFAV_CUDA(cudaLaunchKernel((const void*)k, dim3(blocks), dim3(256), args.data(), 0, st));
    HFAV_LAUNCHED(p->rt, "codegen_rule", st);
    return HFAV_OK;
}

// a part's prepared launch: its stream geometry, compiled kernels and launch shape
struct CgLaunch {
    Stream S;
    cudaKernel_t kern = nullptr, fin = nullptr;
    int CH = 0;
    int64_t strips = 0, nblocks = 0;
    bool ws = false;   // warp strips (placement reg)
    WStrip W;
    int sh = 0;        // warp strips: columns the strips start early
};
// everything of a run that depends only on the plan, the schedule, the
// device and which declared in/out pairs alias: built on the first run of
// that combination, kept with the plan
struct CgPrepared {
    Program G;
    std::vector<CgLaunch> L;
    size_t part_bytes = 0;
};
struct CgCache {
    std::mutex mu;
    std::map<std::string, std::shared_ptr<CgPrepared>> m;
};

static int cg_prepare(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, int dev, CgPrepared* X0) {
    const bool fused = s.fusion != FUSE_UNFUSED;
    const Dag& d = p->dag;
    const hfav_grid& g = p->grids[0];
    const int nx = (int)g.extent[0], ny = (int)g.extent[1];
    const int sms = device_sms();
    Program& G = X0->G;
    int rc = make_program(p, fused, &G);
    if (rc) return rc;
    std::vector<CgLaunch>& L = X0->L;
    L.assign(G.parts.size(), CgLaunch());
    size_t part_bytes = 0;
    const bool inpl = fused && G.parts.size() == 1;
    for (size_t k = 0; k < G.parts.size(); ++k) {
        CgLaunch& X = L[k];
        if ((rc = stream_geometry(p, s, G.parts[k], &X.S))) return rc;
        if (inpl && !X.S.pointwise) mark_inplace(p, &X.S, ax, go);
        const Stream& S = X.S;
        // placement reg: warp strips, unless this run's goal shares its array
        // with an input (the ring kernel saves the bands that run needs)
        if (s.placement == PLACE_REG && std::find(S.inplace.begin(), S.inplace.end(), 1) == S.inplace.end()) {
            if ((rc = wstrip_geometry(p, s, G.parts[k], S, &X.W))) return rc;
            X.ws = true;
            if ((rc = compile(wstrip_source(p, S, G.parts[k], X.W, "hfav_cg_wstrip"), "hfav_cg_wstrip", &X.kern)))
                return rc;
            int per_sm = 0;
            HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)X.kern, X.W.NT, 0));
            const int64_t resident = (int64_t)std::max(1, sms) * std::max(1, per_sm) * (X.W.NT / 32);   // warps
            // strips start sh columns early, so that a lane's cells of the
            // first load sit on vector boundaries (the vector path)
            X.sh = 0;
            if (!S.loads.empty()) {
                const auto ai = std::find(d.axioms.begin(), d.axioms.end(), S.loads[0]);
                X.sh = pmod(caller_view_cg(p, ax[ai - d.axioms.begin()]).org[0] - X.W.HL, X.W.V);
            }
            X.strips = (nx + X.sh + X.W.TXw - 1) / X.W.TXw;
            X.CH = ny;
            double best = 1e300;
            for (int64_t chunks = 1; chunks <= ny; chunks = chunks < 8 ? chunks + 1 : chunks * 5 / 4) {
                const int ch = (int)((ny + chunks - 1) / chunks);
                const int64_t warps = X.strips * ((ny + ch - 1) / ch);
                const double cost = (double)(ch + X.W.fill) * (double)((warps + resident - 1) / resident);
                if (cost < best) { best = cost; X.CH = ch; }
            }
            X.nblocks = (X.strips * ((ny + X.CH - 1) / X.CH) * 32 + X.W.NT - 1) / X.W.NT;
            continue;
        }
        if ((rc = compile(stream_source(p, S, G.parts[k], "hfav_cg_part"), "hfav_cg_part", &X.kern))) return rc;
        // a library kernel takes its attributes per device
        if (S.smem > kSmemDefault)
            HFAV_CUDA(cudaKernelSetAttributeForDevice(X.kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)S.smem + 1024, dev));
        if (!G.fin_reds[k].empty() || !G.fin_rules[k].empty())
            if ((rc = compile(finalize_source(p, G.fin_reds[k], G.fin_rules[k]), "hfav_cg_finalize", &X.fin))) return rc;
        // rows per chunk: the wave count that costs least, each chunk paying
        // the pipeline's fill (yhi - ylo steps beyond its rows)
        int per_sm = 0;
        HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)X.kern, S.NT, S.smem));
        const int64_t resident = (int64_t)std::max(1, sms) * std::max(1, per_sm);
        X.strips = (nx + S.TXc - 1) / S.TXc;
        const int fill = S.yhi - S.ylo;
        X.CH = ny;
        double best = 1e300;
        for (int64_t chunks = 1; chunks <= ny; chunks = chunks < 8 ? chunks + 1 : chunks * 5 / 4) {
            const int ch = (int)((ny + chunks - 1) / chunks);
            const int64_t ctas = X.strips * ((ny + ch - 1) / ch);
            const double cost = (double)(ch + fill) * (double)((ctas + resident - 1) / resident);
            if (cost < best) { best = cost; X.CH = ch; }
        }
        X.nblocks = X.strips * ((ny + X.CH - 1) / X.CH);
        part_bytes = std::max(part_bytes, sizeof(double) * S.reds.size() * (size_t)X.nblocks);
    }
    X0->part_bytes = part_bytes;
    return HFAV_OK;
}

int launch_codegen(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st) {
    const bool fused = s.fusion != FUSE_UNFUSED;
    if (!fused && !has_scalars(p)) return launch_generic(p, ax, go, st);
    const Dag& d = p->dag;
    const hfav_grid& g = p->grids[0];
    const int nx = (int)g.extent[0], ny = (int)g.extent[1];
    int rc = HFAV_OK;
    int dev = 0;
    HFAV_CUDA(cudaGetDevice(&dev));
    // the prepared kernels of this schedule, device and aliasing pattern
    std::string key = std::to_string(dev) + "/" + std::to_string(s.fusion) + "/" + std::to_string(s.placement) + "/" +
                      std::to_string(s.tx) + "x" + std::to_string(s.ty) + "/";
    for (size_t k = 0; k < d.goals.size(); ++k) {
        const int a = k < d.inout.size() ? d.inout[k] : -1;
        key += (a >= 0 && go[k] == ax[a]) ? '1' : '0';
    }
    if (!p->cg_cache) p->cg_cache = std::make_shared<CgCache>();
    CgCache* C = (CgCache*)p->cg_cache.get();
    std::shared_ptr<CgPrepared> prep;
    {
        std::lock_guard<std::mutex> lock(C->mu);
        auto it = C->m.find(key);
        if (it != C->m.end()) prep = it->second;
    }
    if (!prep) {
        auto fresh = std::make_shared<CgPrepared>();
        if ((rc = cg_prepare(p, s, ax, go, dev, fresh.get()))) return rc;
        std::lock_guard<std::mutex> lock(C->mu);
        prep = C->m.emplace(key, fresh).first->second;
    }
    const Program& G = prep->G;
    const std::vector<CgLaunch>& L = prep->L;
    // plan arrays: the fields that cross between parts, over their footprint;
    // the scalars (FP64, by field id); the reductions' partials
    const size_t es = p->dtype == HFAV_F64 ? 8 : 4;
    std::vector<GArr> cross(d.n_fields);
    for (size_t k = 0; k < G.parts.size(); ++k)
        for (int f : L[k].S.crosses) {
            const hfav_field_info& fi = p->an.field[f];
            GArr a;
            const int64_t e0 = nx + fi.halo_lo[0] + fi.halo_hi[0], e1 = ny + fi.halo_lo[1] + fi.halo_hi[1];
            a.pitch[0] = 1; a.pitch[1] = e0; a.pitch[2] = e0 * e1;
            a.org[0] = fi.halo_lo[0]; a.org[1] = fi.halo_lo[1]; a.org[2] = 0;
            a.ext[0] = nx; a.ext[1] = ny; a.ext[2] = 1;
            a.wrap = 0;
            void* ptr;
            if ((rc = scratch(p, "codegen_f" + std::to_string(f), (size_t)(e0 * e1) * es, &ptr))) return rc;
            a.p = ptr;
            cross[f] = a;
        }
    void* scal;
    if ((rc = scratch(p, "codegen_scalars", sizeof(double) * d.n_fields, &scal))) return rc;
    void* part = nullptr;
    if (prep->part_bytes && (rc = scratch(p, "codegen_partials", prep->part_bytes, &part))) return rc;
    for (size_t k = 0; k < G.parts.size(); ++k) {
        const CgLaunch& X = L[k];
        const Stream& S = X.S;
        if (X.ws) {
            ArgPack A;
            for (int f : S.loads) {
                const auto ai = std::find(d.axioms.begin(), d.axioms.end(), f);
                add_array(A, caller_view_cg(p, ax[ai - d.axioms.begin()]));
            }
            for (size_t q = 0; q < S.goals.size(); ++q) {
                GArr y = caller_view_cg(p, go[S.goal_slot[q]]);
                y.wrap = 0;
                add_array(A, y);
            }
            A.add(nx);
            A.add(ny);
            A.add(X.CH);
            A.add((int)X.strips);
            A.add(X.sh);
            auto args = A.ptrs();
            HFAV_CUDA(cudaLaunchKernel((const void*)X.kern, dim3((unsigned)X.nblocks), dim3(X.W.NT), args.data(), 0, st));
            HFAV_LAUNCHED(p->rt, "codegen_fused", st);
            continue;
        }
        ArgPack A;
        for (int f : S.loads) {
            const auto ai = std::find(d.axioms.begin(), d.axioms.end(), f);
            if (ai != d.axioms.end()) add_array(A, caller_view_cg(p, ax[ai - d.axioms.begin()]));
            else add_array(A, cross[f]);
        }
        for (size_t q = 0; q < S.goals.size(); ++q) {
            GArr y = caller_view_cg(p, go[S.goal_slot[q]]);
            y.wrap = 0;
            add_array(A, y);
        }
        for (int f : S.crosses) add_array(A, cross[f]);
        // in/out: save the halo bands of each aliased array before it is overwritten
        for (size_t l = 0; l < S.loads.size(); ++l) {
            if (!S.inplace[l]) continue;
            const SField& F = S.f[S.loads[l]];
            const int HXa = std::max(1, F.hxlo + F.hxhi), HYa = std::max(1, F.hylo + F.hyhi);
            const int64_t chunks = (ny + X.CH - 1) / X.CH;
            const int64_t ncb = X.strips * ((int64_t)ny + F.hylo + F.hyhi) * HXa;
            const int64_t nrb = chunks * HYa * ((int64_t)nx + F.hxlo + F.hxhi);
            void *cb, *rb;
            if ((rc = scratch(p, "inout_cb_" + std::to_string(S.loads[l]), (size_t)ncb * es, &cb))) return rc;
            if ((rc = scratch(p, "inout_rb_" + std::to_string(S.loads[l]), (size_t)nrb * es, &rb))) return rc;
            const auto ai = std::find(d.axioms.begin(), d.axioms.end(), S.loads[l]);
            const GArr src = caller_view_cg(p, ax[ai - d.axioms.begin()]);
            const int rows = ny + F.hylo + F.hyhi, cols = nx + F.hxlo + F.hxhi;
            const int pairs = (int)(X.strips * rows);
            const dim3 gc((pairs + 255) / 256), gr((cols + 255) / 256, (unsigned)(chunks * HYa));
            if (es == 8) {
                inout_colband<double><<<gc, 256, 0, st>>>(src, (double*)cb, nx, ny, S.TXc, F.hxlo, F.hylo, rows, HXa, pairs);
                inout_rowband<double><<<gr, 256, 0, st>>>(src, (double*)rb, nx, ny, X.CH, F.hxlo, F.hylo, cols, HYa);
            } else {
                inout_colband<float><<<gc, 256, 0, st>>>(src, (float*)cb, nx, ny, S.TXc, F.hxlo, F.hylo, rows, HXa, pairs);
                inout_rowband<float><<<gr, 256, 0, st>>>(src, (float*)rb, nx, ny, X.CH, F.hxlo, F.hylo, cols, HYa);
            }
            HFAV_LAUNCHED(p->rt, "codegen_inout_bands", st);
            HFAV_LAUNCHED(p->rt, "codegen_inout_bands", st);
            A.add((const void*)cb);
            A.add((const void*)rb);
        }
        A.add((const void*)scal);
        A.add(part);
        A.add(nx);
        A.add(ny);
        A.add(X.CH);
        auto args = A.ptrs();
        dim3 grd((unsigned)X.strips, (unsigned)((ny + X.CH - 1) / X.CH));
        HFAV_CUDA(cudaLaunchKernel((const void*)X.kern, grd, dim3(S.NT), args.data(), S.smem, st));
        HFAV_LAUNCHED(p->rt, fused ? "codegen_fused" : "codegen_rule", st);
        if (X.fin) {
            ArgPack B;
            B.add((const void*)part);
            B.add((long long)X.nblocks);
            B.add(scal);
            auto bargs = B.ptrs();
            HFAV_CUDA(cudaLaunchKernel((const void*)X.fin, dim3(1), dim3(256), bargs.data(), 0, st));
            HFAV_LAUNCHED(p->rt, "codegen_finalize", st);
        }
    }
    return HFAV_OK;
}

}  // namespace hfav
