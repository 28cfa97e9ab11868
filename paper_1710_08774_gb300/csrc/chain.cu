// chain.cu -- stencil-chain pipelines: the 2D three-stage chain
// (L = 5-pt Laplacian, G = |grad L| / 2, out = G / (1 + G)), the 3D
// four-stage 7-point chain, and the generic one-kernel-per-rule executor.
//
// Fused kernels follow the paper's contraction (Sec. 3.5): one thread per
// column streams along the outer axis (j in 2D, k in 3D) and every
// intermediate lives in a rolling window of 3 rows / planes instead of a full
// array.  The window store is the schedule's placement:
//   reg  -- each thread's own column window in registers, neighbours along
//           the inner axes through one shared row / plane per stage;
//   smem -- the whole 3-row / 3-plane rings in shared memory;
//   hbm  -- the same rings in a per-CTA global-memory slab (L2 resident).
// "sweep" materialises the first stage in HBM and fuses the rest; "unfused"
// runs one kernel per rule over full arrays (launch_generic).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace hfav {

// ---------------------------------------------------------------------------
// generic one-kernel-per-rule executor (the unfused GPU form)
// ---------------------------------------------------------------------------
// Weights reach the kernels in both precisions, rounded on the host: an FP32
// kernel never converts an FP64 parameter on the device (the conversion runs
// on the FP64 pipe, and the compiler may re-derive a weight inside a loop).
template <typename T>
__device__ __forceinline__ T wsel(double d, float f) {
    if constexpr (sizeof(T) == 8) return (T)d;
    else return (T)f;
}

struct GenericArgs {
    int op;
    int nref;
    int ref_arr[27];
    int ref_off[27][3];
    double w[27];
    float wf[27];
    GArr arr[8];
    GArr out;
    int lo[3], n[3];   // iteration region: lo .. lo + n - 1 per axis
};

template <typename T>
__global__ void __launch_bounds__(256) generic_rule_kernel(const GenericArgs a) {
    const int64_t total = (int64_t)a.n[0] * a.n[1] * a.n[2];
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(idx % a.n[0]);
        int64_t rest = idx / a.n[0];
        int j = (int)(rest % a.n[1]);
        int k = (int)(rest / a.n[1]);
        i += a.lo[0]; j += a.lo[1]; k += a.lo[2];
        auto ld = [&](int r) {
            return garr_ld<T>(a.arr[a.ref_arr[r]], i + a.ref_off[r][0], j + a.ref_off[r][1], k + a.ref_off[r][2]);
        };
        T v;
        if (a.op == HFAV_OP_LIMFLUX) {   // in: u(0) u(+1) lap(0) lap(+1)
            const T f = ld(3) - ld(2);
            v = f * (ld(1) - ld(0)) > (T)0 ? (T)0 : f;
        } else if (a.op == HFAV_OP_DIFFUSE) {   // in: u flx(-1) flx(0) fly(-1) fly(0)
            v = ld(0) - wsel<T>(a.w[0], a.wf[0]) * ((ld(2) - ld(1)) + (ld(4) - ld(3)));
        } else if (a.op == HFAV_OP_STENCIL_LINEAR) {
            v = (T)0;
            for (int r = 0; r < a.nref; ++r) {
                T x = garr_ld<T>(a.arr[a.ref_arr[r]], i + a.ref_off[r][0], j + a.ref_off[r][1], k + a.ref_off[r][2]);
                v = r == 0 ? wsel<T>(a.w[r], a.wf[r]) * x : fma(wsel<T>(a.w[r], a.wf[r]), x, v);
            }
        } else if (a.op == HFAV_OP_GRADMAG_HALF) {
            T s = (T)0;
            for (int r = 0; r + 1 < a.nref; r += 2) {
                T x = garr_ld<T>(a.arr[a.ref_arr[r]], i + a.ref_off[r][0], j + a.ref_off[r][1], k + a.ref_off[r][2]);
                T y = garr_ld<T>(a.arr[a.ref_arr[r + 1]], i + a.ref_off[r + 1][0], j + a.ref_off[r + 1][1],
                                 k + a.ref_off[r + 1][2]);
                T d = x - y;
                s = fma(d, d, s);
            }
            v = sqrt(s) * (T)0.5;
        } else {   // SQUASH
            T x = garr_ld<T>(a.arr[a.ref_arr[0]], i + a.ref_off[0][0], j + a.ref_off[0][1], k + a.ref_off[0][2]);
            v = x / ((T)1 + x);
        }
        *garr_ptr<T>(a.out, i, j, k) = v;
    }
}

namespace {

int esize(const hfav_plan_t* p) { return p->dtype == HFAV_F64 ? 8 : 4; }

// view of a caller array of grid 0
GArr caller_view(const hfav_plan_t* p, void* ptr) {
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

}  // namespace

// One kernel per rule, in topological order; intermediates are plan-owned
// full arrays covering their inferred footprint (halo included).
int launch_generic(hfav_plan_t* p, void* const* ax, void* const* go, cudaStream_t st) {
    const Dag& d = p->dag;
    const hfav_grid& g = p->grids[0];
    std::vector<GArr> view(d.n_fields);
    std::vector<char> have(d.n_fields, 0);
    for (size_t k = 0; k < d.axioms.size(); ++k) { view[d.axioms[k]] = caller_view(p, ax[k]); have[d.axioms[k]] = 1; }
    for (size_t k = 0; k < d.goals.size(); ++k) {
        view[d.goals[k]] = caller_view(p, go[k]);
        view[d.goals[k]].wrap = 0;
        have[d.goals[k]] = 1;
    }
    for (int f = 0; f < d.n_fields; ++f) {
        if (have[f] || d.rank[f] == 0) continue;
        const hfav_field_info& fi = p->an.field[f];
        GArr a;
        int64_t e[3];
        for (int x = 0; x < 3; ++x) {
            e[x] = g.extent[x] + fi.halo_lo[x] + fi.halo_hi[x];
            a.org[x] = fi.halo_lo[x];
            a.ext[x] = (int)g.extent[x];
        }
        a.pitch[0] = 1; a.pitch[1] = e[0]; a.pitch[2] = e[0] * e[1];
        a.wrap = 0;
        void* ptr;
        int rc = scratch(p, "generic_f" + std::to_string(f), (size_t)(e[0] * e[1] * e[2]) * esize(p), &ptr);
        if (rc) return rc;
        a.p = ptr;
        view[f] = a;
        have[f] = 1;
    }
    // every read stays inside the array it reads: an input's footprint covers
    // its consumer's region shifted by the offset (axioms of periodic plans wrap)
    for (const Rule& R : d.rules)
        for (const hfav_ref& x : R.in) {
            if (d.rank[x.field] == 0) continue;
            const hfav_field_info &fo = p->an.field[R.out[0]], &fi = p->an.field[x.field];
            const bool wraps = p->bc == HFAV_BC_PERIODIC &&
                               std::find(d.axioms.begin(), d.axioms.end(), x.field) != d.axioms.end();
            for (int a = 0; a < d.ndim && !wraps; ++a)
                if (-fo.halo_lo[a] + x.off[a] < -fi.halo_lo[a] || fo.halo_hi[a] + x.off[a] > fi.halo_hi[a])
                    return set_error(HFAV_EINVAL, "internal: a rule's region leaves its input's footprint");
        }
    for (int r : p->an.order) {
        const Rule& R = d.rules[r];
        GenericArgs a;
        memset(&a, 0, sizeof a);
        a.op = R.op;
        a.nref = (int)R.in.size();
        if (a.nref > 27) return set_error(HFAV_EUNSUPPORTED, "more than 27 refs in one rule");
        std::vector<int> fields;
        for (int k = 0; k < a.nref; ++k) {
            int f = R.in[k].field;
            auto it = std::find(fields.begin(), fields.end(), f);
            int slot = (int)(it - fields.begin());
            if (it == fields.end()) {
                if (fields.size() == 8) return set_error(HFAV_EUNSUPPORTED, "more than 8 input fields in one rule");
                fields.push_back(f);
                a.arr[slot] = view[f];
            }
            a.ref_arr[k] = slot;
            for (int x = 0; x < 3; ++x) a.ref_off[k][x] = R.in[k].off[x];
            a.w[k] = k < (int)R.params.size() ? R.params[k] : 0.0;
        }
        int of = R.out[0];
        a.out = view[of];
        a.out.wrap = 0;
        const hfav_field_info& fo = p->an.field[of];
        for (int x = 0; x < 3; ++x) {
            a.lo[x] = -fo.halo_lo[x];
            a.n[x] = (int)g.extent[x] + fo.halo_lo[x] + fo.halo_hi[x];
        }
        if (R.op == HFAV_OP_EXPR) {   // a user rule body: a generated kernel
            std::vector<int> slot(a.ref_arr, a.ref_arr + a.nref);
            std::vector<GArr> ins(a.arr, a.arr + fields.size());
            int rc = launch_cg_rule(p, R, slot, ins, a.out, a.lo, a.n, st);
            if (rc) return rc;
            continue;
        }
        int64_t total = (int64_t)a.n[0] * a.n[1] * a.n[2];
        int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)device_sms() * 16);
        for (int k = 0; k < 27; ++k) a.wf[k] = (float)a.w[k];
        if (p->dtype == HFAV_F64) generic_rule_kernel<double><<<blocks, 256, 0, st>>>(a);
        else generic_rule_kernel<float><<<blocks, 256, 0, st>>>(a);
        HFAV_LAUNCHED(p->rt, "generic_rule_kernel", st);
    }
    return HFAV_OK;
}

// ---------------------------------------------------------------------------
// 2D chain, fused
// ---------------------------------------------------------------------------
struct C2Args {
    GArr u, out;
    int nx, ny, R;
    double wc, wip, wim, wjp, wjm;   // 5-point star weights
    float fc, fip, fim, fjp, fjm;    // the same, rounded to FP32
    void* slab;                      // hbm placement: per-CTA rings
    int nstrips, sh, vec, vecout;    // reg placement: warp strips, strip origin shift, 16-byte paths
    int nz;                          // COSMO: planes (each on its own)
    double coef;                     // COSMO: c of ustage
    float coeff;                     // the same, rounded to FP32
};

// L at one point from its five star neighbours, summed in the rule's order
template <typename T>
__device__ __forceinline__ T lap5(const C2Args& a, T ip, T im, T jp, T jm, T c) {
    T v = wsel<T>(a.wip, a.fip) * ip;
    v = fma(wsel<T>(a.wim, a.fim), im, v);
    v = fma(wsel<T>(a.wjp, a.fjp), jp, v);
    v = fma(wsel<T>(a.wjm, a.fjm), jm, v);
    return fma(wsel<T>(a.wc, a.fc), c, v);
}

template <typename T>
__device__ __forceinline__ T grad_squash(T lip, T lim, T ljp, T ljm) {
    T gx = lip - lim, gy = ljp - ljm;
    T G = sqrt(fma(gx, gx, gy * gy)) * (T)0.5;
    return G / ((T)1 + G);
}

template <typename T>
__device__ __forceinline__ T ld_u(const C2Args& a, int i, int j) {
    if (!a.u.wrap) {   // halo given: stay inside the allocated halo of 2
        if (i < -2 || i >= a.nx + 2 || j < -2 || j >= a.ny + 2) return (T)0;
    }
    return garr_ld<T>(a.u, i, j, 0);
}

// rows loaded ahead of use by the 2D chain kernels (register queue depth)
#define C2_PD 4

// smem / hbm placement: 3-row rings of u (TX+4 wide) and L (TX+2 wide)
template <typename T, bool HBM>
__global__ void __launch_bounds__(256) chain2d_ring(const C2Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = blockDim.x, t = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * TX;
    const int j0 = (blockIdx.y * blockDim.y + ty) * a.R;
    const int WU = TX + 4, WL = TX + 2;
    const size_t per_group = 3 * WU + 3 * WL;
    T* base;
    if (HBM) {
        size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        base = (T*)a.slab + (cta * blockDim.y + ty) * per_group;
    } else {
        base = (T*)smem_raw + ty * per_group;
    }
    T* su = base;            // [3][WU]
    T* sL = base + 3 * WU;   // [3][WL]
    // row loads C2_PD rows ahead: column t and, for t < 4, column TX + t
    const bool two = t + TX < WU;
    T q[C2_PD], q2[C2_PD];
#pragma unroll
    for (int k = 0; k < C2_PD; ++k) {
        q[k] = ld_u<T>(a, i0 - 2 + t, j0 - 2 + k);
        q2[k] = two ? ld_u<T>(a, i0 - 2 + t + TX, j0 - 2 + k) : (T)0;
    }
    for (int r = j0 - 2; r <= j0 + a.R + 1; ++r) {
        T* ur = su + ((r + 3) % 3) * WU;
        ur[t] = q[0];
        if (two) ur[t + TX] = q2[0];
#pragma unroll
        for (int k = 0; k + 1 < C2_PD; ++k) { q[k] = q[k + 1]; q2[k] = q2[k + 1]; }
        q[C2_PD - 1] = ld_u<T>(a, i0 - 2 + t, r + C2_PD);
        if (two) q2[C2_PD - 1] = ld_u<T>(a, i0 - 2 + t + TX, r + C2_PD);
        __syncthreads();
        if (r >= j0) {   // L(r-1) over columns i0-1 .. i0+TX
            const T* um = su + ((r - 2 + 3) % 3) * WU;
            const T* u0 = su + ((r - 1 + 3) % 3) * WU;
            const T* up = ur;
            T* Lr = sL + ((r - 1 + 3) % 3) * WL;
            for (int c = t; c < WL; c += TX)
                Lr[c] = lap5<T>(a, u0[c + 2], u0[c], up[c + 1], um[c + 1], u0[c + 1]);
        }
        __syncthreads();
        if (r >= j0 + 2) {   // G, out at row r-2
            const int j = r - 2, i = i0 + t;
            const T* Lm = sL + ((r - 3 + 3) % 3) * WL;
            const T* L0 = sL + ((r - 2 + 3) % 3) * WL;
            const T* Lp = sL + ((r - 1 + 3) % 3) * WL;
            T o = grad_squash<T>(L0[t + 2], L0[t], Lp[t + 1], Lm[t + 1]);
            if (i < a.nx && j < a.ny) *garr_ptr<T>(a.out, i, j, 0) = o;
        }
    }
}

// reg placement: warp strips.  Each warp streams a chunk of R rows of a
// strip of 32 V consecutive columns (lane l holds columns s0 + V l ..
// s0 + V l + V - 1) and stores the strip's inner 32 V - 4 columns; strips
// overlap by four columns, so no lane needs data from beyond its strip.  The
// u and L windows (three rows each) are registers, the i-neighbours cross
// lanes by shuffle; no shared memory and no barriers.  Rows are loaded three
// rows ahead; the row loop is unrolled by three so the windows rotate by
// renaming.  Loads and stores are vectors of V cells where a lane's columns
// lie inside the array's rows (the strip origin is shifted so that they are
// aligned), scalars with the periodic wrap elsewhere.

// s / (1 + s) for s = sqrt(g2) / 2, FP32: the equal 1 / (1 + 2 / sqrt(g2))
// with the hardware reciprocal square root and reciprocal (PTX rsqrt.approx
// and rcp.approx, flush-to-zero: relative error a few 2^-23; g2 = 0 or
// subnormal gives 1 / inf = 0)
__device__ __forceinline__ float squash_rsqrt_f32(float g2) {
    float r, o;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(g2));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(o) : "f"(fmaf(2.0f, r, 1.0f)));
    return o;
}

// VW consecutive cells of one lane, loaded and stored as one vector
template <typename T, int VW>
struct alignas(sizeof(T) * VW) VRow {
    static constexpr int V = VW;
    T v[VW];
};

template <typename T>
__device__ __forceinline__ T c2_squash(T gx, T gy) {
    const T g2 = fma(gx, gx, gy * gy);
    if constexpr (sizeof(T) == 4) {
        return squash_rsqrt_f32(g2);
    } else {
        // the same form in FP64: rsqrt (correctly rounded to an ulp) and the
        // refined reciprocal; g2 = 0 gives exactly 0 (tested through the bits)
        const double s = rsqrt(g2);
        return __double_as_longlong(g2) > 0 ? rcp_nr(fma(2.0, s, 1.0)) : 0.0;
    }
}

// one warp's strip; INT: the strip and the two columns on each side lie
// inside the rows and the 16-byte paths are open (no column wrap, no
// per-element fallbacks: the common case, compiled without those branches)
template <typename T, int V, bool INT>
__device__ __forceinline__ void c2w_strip(const C2Args& a, int lane, int s0, int j0) {
    using Row = VRow<T, V>;
    const int c0 = s0 + V * lane;   // first own column
    const bool wrap = a.u.wrap;
    const bool vin = INT || (a.vec && (wrap ? (c0 >= 0 && c0 + V <= a.nx) : (c0 >= -2 && c0 + V <= a.nx + 2)));
    // outputs: columns s0+2 .. s0+32V-3 of the strip that lie in 0 .. nx-1
    const int olo = max(s0 + 2, 0), ohi = min(s0 + 32 * V - 3, a.nx - 1);
    const bool vout = a.vecout && c0 >= olo && c0 + V - 1 <= ohi;
    auto col = [&](const T* ub, int c) -> T {
        if (INT) return ub[c];
        if (wrap) return ub[wrap1(c, a.nx)];
        return (c >= -2 && c < a.nx + 2) ? ub[c] : (T)0;
    };
    // row pointers advance by one pitch per row; under the periodic wrap they
    // are recomputed for rows outside 0 .. ny-1 (rows run over -2 .. ny+1)
    const int64_t pu = a.u.pitch[1], po = a.out.pitch[1];
    const T* row0 = (const T*)a.u.p + (int64_t)a.u.org[1] * pu + a.u.org[0];
    int rl = j0 - 2;   // next row to load
    const T* lp = row0 + (int64_t)(wrap ? wrap1(rl, a.ny) : rl) * pu;
    auto load_next = [&](Row& x) {
        if (vin) {
            x = *(const Row*)(lp + c0);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) x.v[e] = col(lp, c0 + e);
        }
        ++rl;
        lp += pu;
        if (wrap && (rl <= 0 || rl >= a.ny)) lp = row0 + (int64_t)wrap1(rl, a.ny) * pu;
    };
    const T wc = wsel<T>(a.wc, a.fc), wip = wsel<T>(a.wip, a.fip), wim = wsel<T>(a.wim, a.fim);
    const T wjp = wsel<T>(a.wjp, a.fjp), wjm = wsel<T>(a.wjm, a.fjm);
    auto lap = [&](T ip, T im, T jp, T jm, T c) {
        T v = wip * ip;
        v = fma(wim, im, v);
        v = fma(wjp, jp, v);
        v = fma(wjm, jm, v);
        return fma(wc, c, v);
    };
    // rows j0-2 .. rend stream through (step t handles row j0-2+t); out rows j0 .. rend-2
    const int rend = min(j0 + a.R, a.ny) + 1;
    const int n = rend - (j0 - 2) + 1;
    Row Q[3], U[3], L[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) load_next(Q[s]);   // n >= 5: rows j0-2 .. j0 exist
    T* op = (T*)a.out.p + (int64_t)(j0 + a.out.org[1]) * po + a.out.org[0];
    // one step; S = t % 3 (window slot of row t), the flags say which parts run.
    // Lane 0's left and lane 31's right neighbours are its own values (the
    // shuffle's identity): they only reach the columns the strip does not store.
    auto step = [&](auto S, bool pf, bool do_l, bool do_out) {
        constexpr int s = decltype(S)::value, s1 = (s + 1) % 3, s2 = (s + 2) % 3;
        // slots: s holds row r (u) / r-1 (L); s2 row r-1 / r-2; s1 row r-2 / r-3
        U[s] = Q[s];
        if (pf) load_next(Q[s]);
        if (do_l) {   // L at row r-1 from u rows r-2, r-1, r
            const Row& um = U[s1];
            const Row& u0 = U[s2];
            const Row& up = U[s];
            const T left = __shfl_up_sync(0xffffffffu, u0.v[V - 1], 1);
            const T right = __shfl_down_sync(0xffffffffu, u0.v[0], 1);
            Row Lr;
#pragma unroll
            for (int e = 0; e < V; ++e)
                Lr.v[e] = lap(e + 1 < V ? u0.v[e + 1] : right, e > 0 ? u0.v[e - 1] : left, up.v[e], um.v[e], u0.v[e]);
            L[s] = Lr;
        }
        if (do_out) {   // out at row r-2 from L rows r-3, r-2, r-1
            const Row& Lm = L[s1];
            const Row& L0 = L[s2];
            const Row& Lp = L[s];
            const T left = __shfl_up_sync(0xffffffffu, L0.v[V - 1], 1);
            const T right = __shfl_down_sync(0xffffffffu, L0.v[0], 1);
            Row o;
#pragma unroll
            for (int e = 0; e < V; ++e)
                o.v[e] = c2_squash<T>((e + 1 < V ? L0.v[e + 1] : right) - (e > 0 ? L0.v[e - 1] : left),
                                      Lp.v[e] - Lm.v[e]);
            if (vout) {
                *(Row*)(op + c0) = o;
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (c0 + e >= olo && c0 + e <= ohi) op[c0 + e] = o.v[e];
            }
            op += po;
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    // steps 0 .. 5 (n >= 5 always; the prefetch of row t+3 while t+3 < n)
    step(I0{}, 3 < n, false, false);
    step(I1{}, 4 < n, false, false);
    step(I2{}, 5 < n, true, false);
    step(I0{}, 6 < n, true, false);
    step(I1{}, 7 < n, true, true);
    if (5 < n) step(I2{}, 8 < n, true, true);
    int t0 = 6;
    // steady state: whole groups of three steps that all prefetch
    for (; t0 + 2 + 3 < n; t0 += 3) {
        step(I0{}, true, true, true);
        step(I1{}, true, true, true);
        step(I2{}, true, true, true);
    }
    // the last (up to five) steps
    for (; t0 < n; t0 += 3) {
        step(I0{}, t0 + 3 < n, true, true);
        if (t0 + 1 < n) step(I1{}, t0 + 4 < n, true, true);
        if (t0 + 2 < n) step(I2{}, t0 + 5 < n, true, true);
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(256) chain2d_warp(const C2Args a) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31;
    const int64_t wid = ((int64_t)blockIdx.x * (blockDim.x * blockDim.y) + tid) >> 5;
    const int strip = (int)(wid % a.nstrips);
    const int j0 = (int)(wid / a.nstrips) * a.R;
    if (j0 >= a.ny) return;   // whole warp
    // strips overlap by 4 columns: strip k loads 32V columns from s0 and
    // stores the inner 32V - 4
    const int s0 = strip * (32 * V - 4) - 2 - a.sh;
    const bool inside = a.u.wrap ? (s0 >= 0 && s0 + 32 * V <= a.nx) : (s0 >= -2 && s0 + 32 * V <= a.nx + 2);
    if (a.vec && a.vecout && inside) c2w_strip<T, V, true>(a, lane, s0, j0);
    else c2w_strip<T, V, false>(a, lane, s0, j0);
}

// tail of the "sweep" schedule: G and out from a materialised L (halo 1)
template <typename T>
__global__ void __launch_bounds__(256) chain2d_tail(const GArr L, const GArr out, int nx, int ny) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    T o = grad_squash<T>(garr_ld<T>(L, i + 1, j, 0), garr_ld<T>(L, i - 1, j, 0), garr_ld<T>(L, i, j + 1, 0),
                         garr_ld<T>(L, i, j - 1, 0));
    *garr_ptr<T>(out, i, j, 0) = o;
}

namespace {
int rows_per_thread(int64_t cells, int lo, int hi) {
    // enough threads for ~8 warps per SM, at least `lo` rows
    int64_t want = (int64_t)device_sms() * 256;
    int64_t r = cells / want;
    int R = lo;
    while (R < hi && R < r) R *= 2;
    return R;
}
}  // namespace

namespace {
int chunk_planes(int64_t tiles, int nz, int64_t cap, int lead);
}  // namespace

// 2D warp-strip kernel: 16-byte lane vectors for the 32x4 and 64x4 tiles
static inline bool c2w_wide(int TX, int TY) { return TY == 4; }

template <typename T, int V>
static int launch_c2warp(hfav_plan_t* p, C2Args& a, int TX, int TY, cudaStream_t st) {
    const int NT = TX * TY;
    constexpr size_t VB = sizeof(T) * V;   // bytes of one lane's vector
    a.sh = (((a.u.org[0] - 2) % V) + V) % V;   // (s0 + org) a multiple of V
    a.vec = ((uintptr_t)a.u.p % VB == 0) && (a.u.pitch[1] % V == 0);
    a.vecout = ((uintptr_t)a.out.p % VB == 0) && (a.out.pitch[1] % V == 0) && ((a.out.org[0] - a.u.org[0]) % V == 0);
    a.nstrips = (a.nx + a.sh + (32 * V - 4) - 1) / (32 * V - 4);
    static int occ = 0;   // resident CTAs per SM at NT threads (same on every device of the one target)
    static int occ_nt = 0;
    if (occ_nt != NT) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chain2d_warp<T, V>, NT, 0) != cudaSuccess || occ <= 0) {
            cudaGetLastError();
            occ = 1;
        }
        occ_nt = NT;
    }
    // rows per warp: the fewest waves of resident warps times rows (+4 halo rows each)
    a.R = chunk_planes(a.nstrips, a.ny, (int64_t)occ * (NT / 32) * device_sms(), 4);
    const int64_t warps = (int64_t)a.nstrips * ((a.ny + a.R - 1) / a.R);
    const int64_t blocks = (warps + NT / 32 - 1) / (NT / 32);
    chain2d_warp<T, V><<<(unsigned)blocks, dim3(TX, TY), 0, st>>>(a);
    HFAV_LAUNCHED(p->rt, "chain2d_fused", st);
    return HFAV_OK;
}

// ---------------------------------------------------------------------------
// COSMO horizontal diffusion (Sec. 5.3), fused: ulapstage, flux_x, flux_y and
// ustage in one pass with every intermediate in registers.  The same warp
// strips as the 2D chain (a strip of 32 V columns per warp, stores the inner
// 32 V - 4, rows streamed three ahead, i-neighbours by shuffle); each warp
// works in one k plane.  Per arriving u row r: lap at row r-1 (u rows r-2 ..
// r), then flux_y and flux_x at row r-2 (lap rows r-2, r-1), then ustage at
// row r-2 (flux_y rows r-3, r-2); windows of three rows of u, two of lap and
// two of flux_y.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T limflux(T u0, T u1, T l0, T l1) {
    const T f = l1 - l0;
    return f * (u1 - u0) > (T)0 ? (T)0 : f;
}

template <typename T, int V, bool INT>
__device__ __forceinline__ void cosmo_strip(const C2Args& a, int lane, int s0, int j0, int kp) {
    using Row = VRow<T, V>;
    const int c0 = s0 + V * lane;   // first own column
    const bool wrap = a.u.wrap;
    const bool vin = INT || (a.vec && (wrap ? (c0 >= 0 && c0 + V <= a.nx) : (c0 >= -2 && c0 + V <= a.nx + 2)));
    const int olo = max(s0 + 2, 0), ohi = min(s0 + 32 * V - 3, a.nx - 1);
    const bool vout = a.vecout && c0 >= olo && c0 + V - 1 <= ohi;
    auto col = [&](const T* ub, int c) -> T {
        if (INT) return ub[c];
        if (wrap) return ub[wrap1(c, a.nx)];
        return (c >= -2 && c < a.nx + 2) ? ub[c] : (T)0;
    };
    const int64_t pu = a.u.pitch[1], po = a.out.pitch[1];
    const T* row0 = (const T*)a.u.p + (int64_t)(kp + a.u.org[2]) * a.u.pitch[2] + (int64_t)a.u.org[1] * pu + a.u.org[0];
    int rl = j0 - 2;   // next row to load
    const T* lp = row0 + (int64_t)(wrap ? wrap1(rl, a.ny) : rl) * pu;
    auto load_next = [&](Row& x) {
        if (vin) {
            x = *(const Row*)(lp + c0);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) x.v[e] = col(lp, c0 + e);
        }
        ++rl;
        lp += pu;
        if (wrap && (rl <= 0 || rl >= a.ny)) lp = row0 + (int64_t)wrap1(rl, a.ny) * pu;
    };
    const T wc = wsel<T>(a.wc, a.fc), wip = wsel<T>(a.wip, a.fip), wim = wsel<T>(a.wim, a.fim);
    const T wjp = wsel<T>(a.wjp, a.fjp), wjm = wsel<T>(a.wjm, a.fjm), cf = wsel<T>(a.coef, a.coeff);
    auto lap = [&](T ip, T im, T jp, T jm, T c) {
        T v = wip * ip;
        v = fma(wim, im, v);
        v = fma(wjp, jp, v);
        v = fma(wjm, jm, v);
        return fma(wc, c, v);
    };
    const int rend = min(j0 + a.R, a.ny) + 1;
    const int n = rend - (j0 - 2) + 1;
    Row Q[3], U[3], L[3], F[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) load_next(Q[s]);   // n >= 5: rows j0-2 .. j0 exist
    T* op = (T*)a.out.p + (int64_t)(kp + a.out.org[2]) * a.out.pitch[2] + (int64_t)(j0 + a.out.org[1]) * po +
            a.out.org[0];
    // one step; S = t % 3: slot S holds u row r / lap row r-1 / flux_y row r-2,
    // (S+2)%3 the row before each, (S+1)%3 the one before that.  Lane 0's left
    // and lane 31's right neighbours are its own values (the shuffle's
    // identity): they only reach columns the strip does not store.
    auto step = [&](auto Sc, bool pf, bool do_l, bool do_f, bool do_out) {
        constexpr int s = decltype(Sc)::value, s1 = (s + 1) % 3, s2 = (s + 2) % 3;
        U[s] = Q[s];
        if (pf) load_next(Q[s]);
        if (do_l) {   // lap at row r-1 from u rows r-2, r-1, r
            const Row& um = U[s1];
            const Row& u0 = U[s2];
            const Row& up = U[s];
            const T left = __shfl_up_sync(0xffffffffu, u0.v[V - 1], 1);
            const T right = __shfl_down_sync(0xffffffffu, u0.v[0], 1);
            Row Lr;
#pragma unroll
            for (int e = 0; e < V; ++e)
                Lr.v[e] = lap(e + 1 < V ? u0.v[e + 1] : right, e > 0 ? u0.v[e - 1] : left, up.v[e], um.v[e], u0.v[e]);
            L[s] = Lr;
        }
        if (do_f) {   // flux_y and flux_x at row r-2, then ustage there
            const Row& u2 = U[s1];   // u row r-2
            const Row& u1 = U[s2];   // u row r-1
            const Row& l2 = L[s2];   // lap row r-2
            const Row& l1 = L[s];    // lap row r-1
            Row fy, fx;
#pragma unroll
            for (int e = 0; e < V; ++e) fy.v[e] = limflux<T>(u2.v[e], u1.v[e], l2.v[e], l1.v[e]);
            F[s] = fy;
            const T ur = __shfl_down_sync(0xffffffffu, u2.v[0], 1);
            const T lr = __shfl_down_sync(0xffffffffu, l2.v[0], 1);
#pragma unroll
            for (int e = 0; e < V; ++e)
                fx.v[e] = limflux<T>(u2.v[e], e + 1 < V ? u2.v[e + 1] : ur, l2.v[e], e + 1 < V ? l2.v[e + 1] : lr);
            const T fxl = __shfl_up_sync(0xffffffffu, fx.v[V - 1], 1);   // flux_x of the face left of the lane
            if (do_out) {
                const Row& fym = F[s2];   // flux_y row r-3
                Row o;
#pragma unroll
                for (int e = 0; e < V; ++e)
                    o.v[e] = u2.v[e] - cf * ((fx.v[e] - (e > 0 ? fx.v[e - 1] : fxl)) + (fy.v[e] - fym.v[e]));
                if (vout) {
                    *(Row*)(op + c0) = o;
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (c0 + e >= olo && c0 + e <= ohi) op[c0 + e] = o.v[e];
                }
                op += po;
            }
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    // steps 0 .. 5: lap from t = 2, fluxes from t = 3, ustage from t = 4 (n >= 5)
    step(I0{}, 3 < n, false, false, false);
    step(I1{}, 4 < n, false, false, false);
    step(I2{}, 5 < n, true, false, false);
    step(I0{}, 6 < n, true, true, false);
    step(I1{}, 7 < n, true, true, true);
    if (5 < n) step(I2{}, 8 < n, true, true, true);
    int t0 = 6;
    for (; t0 + 2 + 3 < n; t0 += 3) {
        step(I0{}, true, true, true, true);
        step(I1{}, true, true, true, true);
        step(I2{}, true, true, true, true);
    }
    for (; t0 < n; t0 += 3) {
        step(I0{}, t0 + 3 < n, true, true, true);
        if (t0 + 1 < n) step(I1{}, t0 + 4 < n, true, true, true);
        if (t0 + 2 < n) step(I2{}, t0 + 5 < n, true, true, true);
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(256) cosmo_warp(const C2Args a) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31;
    const int64_t wid = ((int64_t)blockIdx.x * (blockDim.x * blockDim.y) + tid) >> 5;
    const int64_t per_plane = (int64_t)a.nstrips * ((a.ny + a.R - 1) / a.R);
    const int kp = (int)(wid / per_plane);
    if (kp >= a.nz) return;   // whole warp
    const int64_t wq = wid - (int64_t)kp * per_plane;
    const int strip = (int)(wq % a.nstrips);
    const int j0 = (int)(wq / a.nstrips) * a.R;
    const int s0 = strip * (32 * V - 4) - 2 - a.sh;
    const bool inside = a.u.wrap ? (s0 >= 0 && s0 + 32 * V <= a.nx) : (s0 >= -2 && s0 + 32 * V <= a.nx + 2);
    if (a.vec && a.vecout && inside) cosmo_strip<T, V, true>(a, lane, s0, j0, kp);
    else cosmo_strip<T, V, false>(a, lane, s0, j0, kp);
}

template <typename T, int V>
static int launch_cosmo_t(hfav_plan_t* p, C2Args& a, int TX, int TY, cudaStream_t st) {
    const int NT = TX * TY;
    constexpr size_t VB = sizeof(T) * V;
    a.sh = (((a.u.org[0] - 2) % V) + V) % V;
    a.vec = ((uintptr_t)a.u.p % VB == 0) && (a.u.pitch[1] % V == 0) && (a.u.pitch[2] % V == 0);
    a.vecout = ((uintptr_t)a.out.p % VB == 0) && (a.out.pitch[1] % V == 0) && (a.out.pitch[2] % V == 0) &&
               ((a.out.org[0] - a.u.org[0]) % V == 0);
    a.nstrips = (a.nx + a.sh + (32 * V - 4) - 1) / (32 * V - 4);
    static int occ = 0, occ_nt = 0;   // resident CTAs per SM at NT threads
    if (occ_nt != NT) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cosmo_warp<T, V>, NT, 0) != cudaSuccess || occ <= 0) {
            cudaGetLastError();
            occ = 1;
        }
        occ_nt = NT;
    }
    a.R = chunk_planes((int64_t)a.nstrips * a.nz, a.ny, (int64_t)occ * (NT / 32) * device_sms(), 4);
    const int64_t warps = (int64_t)a.nstrips * ((a.ny + a.R - 1) / a.R) * a.nz;
    const int64_t blocks = (warps + NT / 32 - 1) / (NT / 32);
    if (blocks > 0x7fffffffLL) return set_error(HFAV_EUNSUPPORTED, "grid too large");
    cosmo_warp<T, V><<<(unsigned)blocks, dim3(TX, TY), 0, st>>>(a);
    HFAV_LAUNCHED(p->rt, "cosmo_fused", st);
    return HFAV_OK;
}

int launch_cosmo(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st) {
    if (s.fusion == FUSE_UNFUSED) return launch_generic(p, ax, go, st);
    if (s.fusion != FUSE_FULL || s.placement != PLACE_REG)
        return set_error(HFAV_EUNSUPPORTED, "the COSMO pipeline runs full:reg or unfused");
    const hfav_grid& g = p->grids[0];
    const ChainMap& m = p->cmap;
    C2Args a;
    memset(&a, 0, sizeof a);
    a.u = caller_view(p, ax[0]);
    a.out = caller_view(p, go[0]);
    a.out.wrap = 0;
    a.nx = (int)g.extent[0]; a.ny = (int)g.extent[1]; a.nz = (int)g.extent[2];
    a.wc = m.w1[13]; a.wip = m.w1[14]; a.wim = m.w1[12]; a.wjp = m.w1[16]; a.wjm = m.w1[10];
    a.fc = (float)a.wc; a.fip = (float)a.wip; a.fim = (float)a.wim; a.fjp = (float)a.wjp; a.fjm = (float)a.wjm;
    a.coef = m.coef;
    a.coeff = (float)m.coef;
    const bool f64 = p->dtype == HFAV_F64, wide = c2w_wide(s.tx, s.ty);
    if (f64) return wide ? launch_cosmo_t<double, 2>(p, a, s.tx, s.ty, st) : launch_cosmo_t<double, 1>(p, a, s.tx, s.ty, st);
    return wide ? launch_cosmo_t<float, 4>(p, a, s.tx, s.ty, st) : launch_cosmo_t<float, 2>(p, a, s.tx, s.ty, st);
}

int launch_chain2d(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st) {
    if (s.fusion == FUSE_UNFUSED) return launch_generic(p, ax, go, st);
    const hfav_grid& g = p->grids[0];
    const ChainMap& m = p->cmap;
    const int nx = (int)g.extent[0], ny = (int)g.extent[1];
    C2Args a;
    memset(&a, 0, sizeof a);
    a.u = caller_view(p, ax[0]);
    a.out = caller_view(p, go[0]);
    a.out.wrap = 0;
    a.nx = nx; a.ny = ny;
    a.wc = m.w1[13]; a.wip = m.w1[14]; a.wim = m.w1[12]; a.wjp = m.w1[16]; a.wjm = m.w1[10];
    a.fc = (float)a.wc; a.fip = (float)a.wip; a.fim = (float)a.wim; a.fjp = (float)a.wjp; a.fjm = (float)a.wjm;
    for (int k = 0; k < 27; ++k)
        if (k != 13 && k != 14 && k != 12 && k != 16 && k != 10 && m.w1[k] != 0.0)
            return set_error(HFAV_EUNSUPPORTED, "fused 2D chain takes a 5-point star stencil");
    const bool f64 = p->dtype == HFAV_F64;
    const size_t es = esize(p);
    if (s.fusion == FUSE_SWEEP) {
        // stage 1 materialised over its footprint (generic kernel), stages 2-3 fused
        hfav_plan_t& P = *p;
        const Rule& R0 = P.dag.rules[m.rules[0]];
        int Lf = R0.out[0];
        const hfav_field_info& fi = P.an.field[Lf];
        GArr L;
        int64_t ex = nx + fi.halo_lo[0] + fi.halo_hi[0], ey = ny + fi.halo_lo[1] + fi.halo_hi[1];
        void* ptr;
        int rc = scratch(p, "chain_L", (size_t)(ex * ey) * es, &ptr);
        if (rc) return rc;
        L.p = ptr; L.pitch[0] = 1; L.pitch[1] = ex; L.pitch[2] = ex * ey;
        L.org[0] = fi.halo_lo[0]; L.org[1] = fi.halo_lo[1]; L.org[2] = 0;
        L.ext[0] = nx; L.ext[1] = ny; L.ext[2] = 1; L.wrap = 0;
        GenericArgs ga;
        memset(&ga, 0, sizeof ga);
        ga.op = HFAV_OP_STENCIL_LINEAR;
        ga.nref = (int)R0.in.size();
        ga.arr[0] = a.u;
        for (int k = 0; k < ga.nref; ++k) {
            ga.ref_arr[k] = 0;
            for (int x = 0; x < 3; ++x) ga.ref_off[k][x] = R0.in[k].off[x];
            ga.w[k] = R0.params[k];
        }
        ga.out = L;
        ga.lo[0] = -fi.halo_lo[0]; ga.lo[1] = -fi.halo_lo[1]; ga.lo[2] = 0;
        ga.n[0] = (int)ex; ga.n[1] = (int)ey; ga.n[2] = 1;
        int blocks = (int)std::min<int64_t>((ex * ey + 255) / 256, (int64_t)device_sms() * 16);
        for (int k = 0; k < 27; ++k) ga.wf[k] = (float)ga.w[k];
        if (f64) generic_rule_kernel<double><<<blocks, 256, 0, st>>>(ga);
        else generic_rule_kernel<float><<<blocks, 256, 0, st>>>(ga);
        HFAV_LAUNCHED(p->rt, "generic_rule_kernel", st);
        dim3 blk(s.tx, s.ty), grd((nx + s.tx - 1) / s.tx, (ny + s.ty - 1) / s.ty);
        if (f64) chain2d_tail<double><<<grd, blk, 0, st>>>(L, a.out, nx, ny);
        else chain2d_tail<float><<<grd, blk, 0, st>>>(L, a.out, nx, ny);
        HFAV_LAUNCHED(p->rt, "chain2d_tail", st);
        return HFAV_OK;
    }
    // full fusion
    a.R = rows_per_thread((int64_t)nx * ny, 8, 64);
    const int TX = s.tx, TY = s.ty;
    dim3 blk(TX, TY);
    dim3 grd((nx + TX - 1) / TX, (ny + a.R * TY - 1) / (a.R * TY));
    if (s.placement == PLACE_REG) {
        // cells per lane: 16-byte vectors for the 32x4 / 64x4 tiles, half that
        // (fewer registers, more resident warps) for 128x2 / 32x8
        const bool wide = c2w_wide(TX, TY);
        if (f64) return wide ? launch_c2warp<double, 2>(p, a, TX, TY, st) : launch_c2warp<double, 1>(p, a, TX, TY, st);
        return wide ? launch_c2warp<float, 4>(p, a, TX, TY, st) : launch_c2warp<float, 2>(p, a, TX, TY, st);
    }
    if (s.placement == PLACE_SMEM) {
        size_t sm = (size_t)TY * (3 * (TX + 4) + 3 * (TX + 2)) * es;
        if (f64) chain2d_ring<double, false><<<grd, blk, sm, st>>>(a);
        else chain2d_ring<float, false><<<grd, blk, sm, st>>>(a);
    } else {
        size_t per = (size_t)TY * (3 * (TX + 4) + 3 * (TX + 2)) * es;
        void* slab;
        int rc = scratch(p, "chain2d_slab", per * grd.x * grd.y, &slab);
        if (rc) return rc;
        a.slab = slab;
        if (f64) chain2d_ring<double, true><<<grd, blk, 0, st>>>(a);
        else chain2d_ring<float, true><<<grd, blk, 0, st>>>(a);
    }
    HFAV_LAUNCHED(p->rt, "chain2d_fused", st);
    return HFAV_OK;
}

// ---------------------------------------------------------------------------
// 3D chain, fused: s1 = D7(u), s2 = D7(s1), s3 = |grad s2| / 2, out = s3/(1+s3)
// CTA tile TX x TY columns in (i, j); each thread streams k over a chunk.
// Planes: u on (TX+6)(TY+6), s1 on (TX+4)(TY+4), s2 on (TX+2)(TY+2).
// ---------------------------------------------------------------------------
struct C3Args {
    GArr u, out;
    int nx, ny, nz, K;
    double a1[7], a2[7];   // weights: centre, +i, -i, +j, -j, +k, -k
    float f1[7], f2[7];    // the same, rounded to FP32
    void* slab;
    unsigned* err;         // set when a bounded wait on a copy gave up (the plan's timeout word)
};

template <typename T>
__device__ __forceinline__ T ld_u3(const C3Args& a, int i, int j, int k) {
    if (!a.u.wrap) {
        if (i < -3 || i >= a.nx + 3 || j < -3 || j >= a.ny + 3 || k < -3 || k >= a.nz + 3) return (T)0;
    }
    return garr_ld<T>(a.u, i, j, k);
}

template <typename T>
__device__ __forceinline__ T d7(const double* w, const float* f, T ip, T im, T jp, T jm, T kp, T km, T c) {
    T v = wsel<T>(w[1], f[1]) * ip;
    v = fma(wsel<T>(w[2], f[2]), im, v);
    v = fma(wsel<T>(w[3], f[3]), jp, v);
    v = fma(wsel<T>(w[4], f[4]), jm, v);
    v = fma(wsel<T>(w[5], f[5]), kp, v);
    v = fma(wsel<T>(w[6], f[6]), km, v);
    return fma(wsel<T>(w[0], f[0]), c, v);
}

// ring placement (smem or hbm): 3 planes of u, s1, s2 per CTA
template <typename T, bool HBM>
__global__ void __launch_bounds__(256) chain3d_ring(const C3Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = blockDim.x, TY = blockDim.y, NT = TX * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * a.K;
    const int PU = (TX + 6) * (TY + 6), P1 = (TX + 4) * (TY + 4), P2 = (TX + 2) * (TY + 2);
    T* base;
    if (HBM) {
        size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        base = (T*)a.slab + cta * (size_t)(3 * (PU + P1 + P2));
    } else {
        base = (T*)smem_raw;
    }
    T* su = base;            // [3][PU]
    T* s1 = su + 3 * PU;     // [3][P1]
    T* s2 = s1 + 3 * P1;     // [3][P2]
    // plane kk of u is needed for kk in [k0-3, k0+K+2]
    for (int kk = k0 - 3; kk <= k0 + a.K + 2; ++kk) {
        T* up = su + ((kk + 6) % 3) * PU;
        for (int c = tid; c < PU; c += NT) {
            int ci = c % (TX + 6), cj = c / (TX + 6);
            up[c] = ld_u3<T>(a, i0 - 3 + ci, j0 - 3 + cj, kk);
        }
        __syncthreads();
        if (kk >= k0 - 1) {   // s1 plane kk-1 on (TX+4)(TY+4)
            const int kq = kk - 1;
            const T* um = su + ((kq - 1 + 6) % 3) * PU;
            const T* u0 = su + ((kq + 6) % 3) * PU;
            const T* uq = up;
            T* o = s1 + ((kq + 6) % 3) * P1;
            for (int c = tid; c < P1; c += NT) {
                int ci = c % (TX + 4) + 1, cj = c / (TX + 4) + 1;   // position in the u tile
                int q = cj * (TX + 6) + ci;
                o[c] = d7<T>(a.a1, a.f1, u0[q + 1], u0[q - 1], u0[q + TX + 6], u0[q - TX - 6], uq[q], um[q], u0[q]);
            }
        }
        __syncthreads();
        if (kk >= k0 + 1) {   // s2 plane kk-2 on (TX+2)(TY+2)
            const int kq = kk - 2;
            const T* pm = s1 + ((kq - 1 + 6) % 3) * P1;
            const T* p0 = s1 + ((kq + 6) % 3) * P1;
            const T* pp = s1 + ((kq + 1 + 6) % 3) * P1;
            T* o = s2 + ((kq + 6) % 3) * P2;
            for (int c = tid; c < P2; c += NT) {
                int ci = c % (TX + 2) + 1, cj = c / (TX + 2) + 1;
                int q = cj * (TX + 4) + ci;
                o[c] = d7<T>(a.a2, a.f2, p0[q + 1], p0[q - 1], p0[q + TX + 4], p0[q - TX - 4], pp[q], pm[q], p0[q]);
            }
        }
        __syncthreads();
        if (kk >= k0 + 3) {   // out plane kk-3
            const int kq = kk - 3;
            const T* qm = s2 + ((kq - 1 + 6) % 3) * P2;
            const T* q0 = s2 + ((kq + 6) % 3) * P2;
            const T* qp = s2 + ((kq + 1 + 6) % 3) * P2;
            const int ti = threadIdx.x, tj = threadIdx.y;
            const int q = (tj + 1) * (TX + 2) + ti + 1;
            T gx = q0[q + 1] - q0[q - 1], gy = q0[q + TX + 2] - q0[q - TX - 2], gz = qp[q] - qm[q];
            T s3 = sqrt(fma(gx, gx, fma(gy, gy, gz * gz))) * (T)0.5;
            int i = i0 + ti, j = j0 + tj;
            if (i < a.nx && j < a.ny && kq < a.nz) *garr_ptr<T>(a.out, i, j, kq) = s3 / ((T)1 + s3);
        }
    }
}

// register-window form (placement reg).  The CTA's TX x TY threads own an
// output tile of TX x TYO cells (TYO = 16; 8 for TY = 2, which keeps the
// per-thread windows of the widest tile within the register file) and
// stream k.  Every stage plane (u, s1, s2) is a W x R array in shared memory
// with one width W = TX + 8 and one column numbering (column c <-> i = i0 -
// 3 + c, stored at row * W + c + 1), so a stage evaluates its whole plane as
// dense pairs of adjacent cells: pair q is stored at 2q, 2q + 1 and reads its
// input plane around 2q + W (the input row below).  No index arithmetic per
// position, 8-byte (FP32) or 16-byte (FP64) shared accesses, and no bank
// conflicts from rows of different widths.  Columns outside the loaded u
// columns produce meaningless s1 / s2 values that no valid cell reads: s1 is
// valid on columns 1 .. TX+4, s2 on 2 .. TX+3, and out takes 3 .. TX+2.
// Each stage keeps the k window (three planes) of its input at its own
// pairs in registers; the window's middle plane is also the centre of the
// in-plane stencil, so only the four in-plane neighbours go through shared
// memory.
template <int TX, int TY>
struct C3Tile {
    static constexpr int NT = TX * TY, M = (TY >= 4 ? 16 : 8) / TY, TYO = TY * M;
    static constexpr int W = TX + 8, WL = TX + 6;   // row stride; loaded u columns
    static constexpr int RU = TYO + 6, R1 = TYO + 4, R2 = TYO + 2;
    static constexpr int PU = W * RU, P1 = W * R1, P2 = W * R2;
    static constexpr int LU = WL * RU, NU = (LU + NT - 1) / NT;   // u elements loaded per plane
    static constexpr int Q1 = P1 / 2, Q2 = P2 / 2, QO = TX * TYO / 2;   // pairs per stage
    static constexpr int N1 = (Q1 + NT - 1) / NT, N2 = (Q2 + NT - 1) / NT, NO = QO / NT;
    static_assert(QO % NT == 0 && TX % 2 == 0, "output pairs split evenly over the threads");
    // u planes are fetched ND planes ahead with asynchronous copies into a
    // ring of ND + 2 plane buffers (the s1 stage reads planes kk-1 and kk)
    static constexpr int ND = 2, NB = ND + 2;
    // TMA form: cells of a periodic edge tile patched per thread (one i band
    // of 4 columns and one j band of 3 rows at most)
    static constexpr int NF = (3 * W + 4 * RU + NT - 1) / NT;
    static constexpr size_t smem(size_t es) { return (size_t)(NB * PU + 3 * P1 + 3 * P2) * es; }
    // TMA form: u plane slots padded to 128 bytes (copy destinations), the
    // NB completion barriers after the rings, 128 bytes to align the base
    static constexpr int pua(size_t es) { return (int)(((size_t)PU * es + 127) / 128 * 128 / es); }
    static constexpr size_t smem_tma(size_t es) {
        return (size_t)(NB * pua(es) + 3 * P1 + 3 * P2) * es + NB * 8 + 128;
    }
};

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

// asynchronous global -> shared copy of one element (cp.async, cached in L1)
template <int BYTES>
__device__ __forceinline__ void cp_async_el(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// the same star summed as a tree of pairs (three dependent steps instead of
// seven), for the FP32 quad kernel: a different rounding order, within the
// FP32 bar
__device__ __forceinline__ float pt7t(const float* w, float ip, float im, float jp, float jm, float kp, float km,
                                      float c) {
    const float a = fmaf(w[2], im, w[1] * ip);
    const float b = fmaf(w[4], jm, w[3] * jp);
    const float d = fmaf(w[6], km, w[5] * kp);
    return fmaf(w[0], c, a) + (b + d);
}

// one 7-point star in the rule's summation order (+i, -i, +j, -j, +k, -k, centre)
template <typename T>
__device__ __forceinline__ T pt7(const T* w, T ip, T im, T jp, T jm, T kp, T km, T c) {
    T v = w[1] * ip;
    v = fma(w[2], im, v);
    v = fma(w[3], jp, v);
    v = fma(w[4], jm, v);
    v = fma(w[5], kp, v);
    v = fma(w[6], km, v);
    return fma(w[0], c, v);
}

// out = s3 / (1 + s3), s3 = sqrt(g2) / 2.  FP64 evaluates that quotient as
// written (IEEE square root and division); FP32 takes the equal form
// 1 / (1 + 2 / sqrt(g2)) (squash_rsqrt_f32).
template <typename T>
__device__ __forceinline__ T chain3_out(T gx, T gy, T gz) {
    const T g2 = fma(gx, gx, fma(gy, gy, gz * gz));
    if constexpr (sizeof(T) == 4) {
        return squash_rsqrt_f32(g2);
    } else {
        const T s3 = sqrt(g2) * (T)0.5;
        return s3 / ((T)1 + s3);
    }
}

// LOAD selects how u planes reach shared memory: 0, one cp.async per element
// (any layout); 1, the tensor memory accelerator -- one tiled tensor copy of
// the whole W x RU plane tile per plane, completed on one mbarrier per ring
// slot, with the cells a periodic edge tile wraps to patched from registers
// after the copy lands.  The host takes LOAD 1 only where the copy is
// 16-byte aligned and a tile touches at most one edge per axis (see
// launch_c3regw).
template <typename T, int TX, int TY, int LOAD>
__global__ void __launch_bounds__(TX * TY) chain3d_regw(const C3Args a, const __grid_constant__ CUtensorMap tmap) {
    using G = C3Tile<TX, TY>;
    using V = typename Pair<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sbase = smem_raw;
    if constexpr (LOAD == 1) sbase += (128u - (smem_u32(smem_raw) & 127u)) & 127u;
    constexpr int PUS = LOAD == 1 ? G::pua(sizeof(T)) : G::PU;   // stride of the u plane slots
    T* U = (T*)sbase;             // [NB][PUS] ring of u planes
    T* S1 = U + G::NB * PUS;      // [3][P1] ring of s1 planes
    T* S2 = S1 + 3 * G::P1;       // [3][P2] ring of s2 planes
    unsigned long long* bars = (unsigned long long*)(S2 + 3 * G::P2);   // LOAD 1: one per u slot
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * G::TYO, k0 = blockIdx.z * a.K;
    const T* u = (const T*)a.u.p;
    // loaded u elements: in-plane global offset (wrapped / halo-given;
    // 32-bit, a padded plane is far below 2^31 elements) and shared offset
    constexpr int NUL = LOAD == 0 ? G::NU : 1;
    int gu[NUL], su[NUL];
    // LOAD 1 on a periodic grid: a tile on the i or j edge gets from its
    // box the out-of-range cells of the plane tile as zeros (or as the
    // array's unread halo); those cells -- three rows of the j edge, four
    // columns of the i edge -- are patched with their wrapped values, which
    // each thread (up to G::NF cells) loads two planes ahead into registers
    // and stores once the plane's copy has landed
    const bool iedge = a.u.wrap && (i0 == 0 || i0 + TX >= a.nx);
    const bool jedge = a.u.wrap && (j0 == 0 || j0 + G::TYO >= a.ny);
    const bool patch = LOAD == 1 && (iedge || jedge);
    int pso[G::NF];       // patched cell: shared offset in the plane slot (-1: none)
    int pgo[G::NF];       // its wrapped in-plane global offset
    T pv0[G::NF], pv1[G::NF], pv2[G::NF];   // its values for planes it, it + 1, it + 2
    bool timed_out = false;
    if constexpr (LOAD == 1) {
        const int nj = jedge ? 3 : 0, ni = iedge ? 4 : 0;
        const int rj0 = j0 == 0 ? 0 : G::RU - 3;         // rows of the j band
        const int ci0 = i0 == 0 ? 0 : G::W - 4;          // columns of the i band
        const int ro0 = (jedge && j0 == 0) ? 3 : 0;      // first row outside the j band
        const int ncell = nj * G::W + ni * (G::RU - nj);
#pragma unroll
        for (int f = 0; f < G::NF; ++f) {
            const int e = tid + f * G::NT;
            pso[f] = -1;
            pgo[f] = 0;
            pv0[f] = pv1[f] = pv2[f] = (T)0;
            if (!patch || e >= ncell) continue;
            int r, c;
            if (e < nj * G::W) { r = rj0 + e / G::W; c = e % G::W; }
            else { const int q = e - nj * G::W; r = ro0 + q / 4; c = ci0 + q % 4; }
            const int gi = wrap_idx(i0 - 4 + c, a.nx), gj = wrap_idx(j0 - 3 + r, a.ny);
            pso[f] = r * G::W + c;
            pgo[f] = (int)((int64_t)(gj + a.u.org[1]) * a.u.pitch[1] + (gi + a.u.org[0]));
        }
        if (tid == 0) {
            for (int b = 0; b < G::NB; ++b) mbar_init(bars + b, 1);
            mbar_init_fence();
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < (LOAD == 0 ? G::NU : 0); ++r) {
        const int e = min(tid + r * G::NT, G::LU - 1);
        const int row = e / G::WL, col = e - row * G::WL;
        int gi = i0 - 3 + col, gj = j0 - 3 + row;
        if (a.u.wrap) {
            gi = wrap_idx(gi, a.nx);
            gj = wrap_idx(gj, a.ny);
        } else {
            gi = min(max(gi, -3), a.nx + 2);
            gj = min(max(gj, -3), a.ny + 2);
        }
        gu[r] = (int)((int64_t)(gj + a.u.org[1]) * a.u.pitch[1] + (gi + a.u.org[0]));
        su[r] = row * G::W + col + 1;
    }
    // output pairs: pair o = tid + r NT is row o / (TX/2), columns 3 + 2 (o % (TX/2)) and the next
    T* op[G::NO];
    int bo[G::NO];
    bool ok0[G::NO], ok1[G::NO];
#pragma unroll
    for (int r = 0; r < G::NO; ++r) {
        const int o = tid + r * G::NT;
        const int row = o / (TX / 2), pc = o - row * (TX / 2);
        const int i = i0 + 2 * pc, j = j0 + row;
        ok0[r] = i < a.nx && j < a.ny;
        ok1[r] = i + 1 < a.nx && j < a.ny;
        op[r] = garr_ptr<T>(a.out, min(i, a.nx - 1), min(j, a.ny - 1), min(k0, a.nz - 1));
        bo[r] = (row + 1) * G::W + 4 + 2 * pc;
    }
    V wu[G::N1][3], w1[G::N2][3], w2[G::NO][3];
    const V zero = {(T)0, (T)0};
#pragma unroll
    for (int r = 0; r < G::N1; ++r) wu[r][0] = wu[r][1] = wu[r][2] = zero;
#pragma unroll
    for (int r = 0; r < G::N2; ++r) w1[r][0] = w1[r][1] = w1[r][2] = zero;
#pragma unroll
    for (int r = 0; r < G::NO; ++r) w2[r][0] = w2[r][1] = w2[r][2] = zero;
    T wa[7], wb[7];
#pragma unroll
    for (int x = 0; x < 7; ++x) {
        wa[x] = wsel<T>(a.a1[x], a.f1[x]);
        wb[x] = wsel<T>(a.a2[x], a.f2[x]);
    }
    // Skewed pipeline with one barrier per plane: iteration it loads the u
    // plane kk = k0 - 3 + it and computes s1 at plane kk-1, s2 at kk-3 and
    // out at kk-5, so every stage reads only planes written in earlier
    // iterations.  u planes sit in a ring of NB slots (slot it % NB), s1 and
    // s2 planes in rings of three (the plane made at iteration it in slot
    // it % 3).
    const int nu = a.K + 6, nit = a.K + 8;
    const int64_t kstep = a.out.pitch[2];
    auto fetch = [&](int it) {
        if constexpr (LOAD == 0) {
            if (it < nu) {
                const int kk = k0 - 3 + it;
                const int kw = a.u.wrap ? wrap1(kk, a.nz) : min(max(kk, -3), a.nz + 2);
                const T* ub = u + (int64_t)(kw + a.u.org[2]) * a.u.pitch[2];
                T* Ub = U + (it % G::NB) * PUS;
#pragma unroll
                for (int r = 0; r < G::NU; ++r)
                    if (r < G::NU - 1 || tid + r * G::NT < G::LU) cp_async_el<sizeof(T)>(Ub + su[r], ub + gu[r]);
            }
            cp_async_commit();   // one group per plane, empty past the chunk's end
        } else {
            if (it >= nu) return;
            const int kk = k0 - 3 + it;
            const int kw = a.u.wrap ? wrap1(kk, a.nz) : min(max(kk, -3), a.nz + 2);
            if (tid == 0) {
                T* Ub = U + (it % G::NB) * PUS;
                unsigned long long* bar = bars + it % G::NB;
                // the slot's previous plane was read before the barrier this
                // thread just passed; order those reads before the copy's writes
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, (unsigned)(G::PU * sizeof(T)));
                // column i0 - 4 + c at c, row j0 - 3 + r at r: the W x RU plane tile
                tma_load_3d(Ub, &tmap, i0 - 4 + a.u.org[0], j0 - 3 + a.u.org[1], kw + a.u.org[2], bar);
            }
            if (patch) {   // wrapped cells of plane it, two planes ahead of their use
                const T* pl = u + (int64_t)(kw + a.u.org[2]) * a.u.pitch[2];
#pragma unroll
                for (int f = 0; f < G::NF; ++f)
                    if (pso[f] >= 0) pv2[f] = pl[pgo[f]];
            }
        }
    };
    static_assert(G::ND == 2, "the patch registers hold two planes ahead");
    fetch(0);
    if constexpr (LOAD == 1) {
#pragma unroll
        for (int f = 0; f < G::NF; ++f) pv0[f] = pv2[f];
    }
    fetch(1);
    if constexpr (LOAD == 1) {
#pragma unroll
        for (int f = 0; f < G::NF; ++f) pv1[f] = pv2[f];
    }
    int c0 = 0, c1 = 1, c2 = 2;   // it % 3, (it + 1) % 3, (it + 2) % 3
    for (int it = 0; it < nit; ++it) {
        if constexpr (LOAD == 0) {
            cp_async_wait<G::ND - 1>();   // this thread's copies of plane it are done
        } else if (it < nu) {
            if (!mbar_wait_bounded(bars + it % G::NB, (unsigned)(it / G::NB) & 1u, a.err)) timed_out = true;
            if (patch) {   // the copy has landed: overwrite its out-of-range cells
                T* Ub = U + (it % G::NB) * PUS;
#pragma unroll
                for (int f = 0; f < G::NF; ++f)
                    if (pso[f] >= 0) Ub[pso[f]] = pv0[f];
            }
        }
        __syncthreads();
        // the slot of plane it + ND held plane it - 2, last read at it - 1
        fetch(it + G::ND);
        // the planes this iteration reads and writes: distinct ring slots, so
        // the stages' shared loads may move ahead of earlier stages' stores
        const T* __restrict__ Ub = U + (it % G::NB) * PUS;
        const T* __restrict__ Up = U + ((it + G::NB - 1) % G::NB) * PUS;
        T* __restrict__ S1b = S1 + c0 * G::P1;
        const T* __restrict__ S1n = S1 + c2 * G::P1;
        const T* __restrict__ S1p = S1 + c1 * G::P1;
        T* __restrict__ S2b = S2 + c0 * G::P2;
        const T* __restrict__ S2n = S2 + c2 * G::P2;
        const T* __restrict__ S2p = S2 + c1 * G::P2;
        // s1 at plane kk-1: window u(kk-2 .. kk), in-plane neighbours from u(kk-1)
        if (it < nu) {
            const bool comp = it >= 2;
#pragma unroll
            for (int r = 0; r < G::N1; ++r) {
                const int q = tid + r * G::NT;
                if (r == G::N1 - 1 && q >= G::Q1) continue;
                const int b = 2 * q + G::W;
                wu[r][0] = wu[r][1]; wu[r][1] = wu[r][2]; wu[r][2] = *(const V*)(Ub + b);
                if (!comp) continue;
                const V n = *(const V*)(Up + b + G::W), sth = *(const V*)(Up + b - G::W);
                const T l = Up[b - 1], rt = Up[b + 2];
                const V c = wu[r][1];
                V o;
                o.x = pt7<T>(wa, c.y, l, n.x, sth.x, wu[r][2].x, wu[r][0].x, c.x);
                o.y = pt7<T>(wa, rt, c.x, n.y, sth.y, wu[r][2].y, wu[r][0].y, c.y);
                *(V*)(S1b + 2 * q) = o;
            }
        }
        // s2 at plane kk-3 from the s1 planes kk-2 (window push, made at
        // it-1) and kk-3 (in-plane, made at it-2); s1 exists from plane
        // k0-2 (it = 3) to k0+K+1 (it = K+6)
        if (it >= 3 && it < nu + 1) {
            const bool comp = it >= 5;
#pragma unroll
            for (int r = 0; r < G::N2; ++r) {
                const int q = tid + r * G::NT;
                if (r == G::N2 - 1 && q >= G::Q2) continue;
                const int b = 2 * q + G::W;
                w1[r][0] = w1[r][1]; w1[r][1] = w1[r][2]; w1[r][2] = *(const V*)(S1n + b);
                if (!comp) continue;
                const V n = *(const V*)(S1p + b + G::W), sth = *(const V*)(S1p + b - G::W);
                const T l = S1p[b - 1], rt = S1p[b + 2];
                const V c = w1[r][1];
                V o;
                o.x = pt7<T>(wb, c.y, l, n.x, sth.x, w1[r][2].x, w1[r][0].x, c.x);
                o.y = pt7<T>(wb, rt, c.x, n.y, sth.y, w1[r][2].y, w1[r][0].y, c.y);
                *(V*)(S2b + 2 * q) = o;
            }
        }
        // out at plane kk-5 from the s2 planes kk-4 (window push, made at
        // it-1) and kk-5 (in-plane, made at it-2); s2 exists from plane k0-1 (it = 6)
        if (it >= 6) {
            const bool store = it >= 8 && k0 - 8 + it < a.nz;
#pragma unroll
            for (int r = 0; r < G::NO; ++r) {
                const int b = bo[r];
                w2[r][0] = w2[r][1]; w2[r][1] = w2[r][2]; w2[r][2] = *(const V*)(S2n + b);
                if (it >= 8) {
                    const V n = *(const V*)(S2p + b + G::W), sth = *(const V*)(S2p + b - G::W);
                    const T l = S2p[b - 1], rt = S2p[b + 2];
                    const V c = w2[r][1];
                    const T x0 = chain3_out<T>(c.y - l, n.x - sth.x, w2[r][2].x - w2[r][0].x);
                    const T x1 = chain3_out<T>(rt - c.x, n.y - sth.y, w2[r][2].y - w2[r][0].y);
                    if (store) {
                        if (ok0[r]) op[r][0] = x0;
                        if (ok1[r]) op[r][1] = x1;
                    }
                    op[r] += kstep;
                }
            }
        }
        const int t = c0; c0 = c1; c1 = c2; c2 = t;
        if constexpr (LOAD == 1) {
#pragma unroll
            for (int f = 0; f < G::NF; ++f) { pv0[f] = pv1[f]; pv1[f] = pv2[f]; }
        }
    }
    if constexpr (LOAD == 1) {
        // after a timed-out wait, give the copies still in flight (the last
        // plane of each slot) a bounded time to land before the CTA exits
        if (timed_out)
            for (int it = max(0, nu - G::NB); it < nu; ++it)
                mbar_wait_bounded(bars + it % G::NB, (unsigned)(it / G::NB) & 1u, nullptr);
    }
}

// FP32 register-window form on quads.  The same plane tiles, rings, skewed
// pipeline and TMA staging as chain3d_regw (LOAD 1), with each thread
// evaluating a stage on quads of four adjacent cells (16-byte shared loads
// and stores, one pair of scalar i-neighbour loads per four cells) and the
// plane loop unrolled by three so that the k windows, the s1 / s2 ring
// slots and the patch registers rotate by index instead of by copies.
// Output quads are stored as 16-byte vectors.  Taken for FP32 where the TMA
// copy applies (the host's c3_tma_ok), which also makes every output quad
// whole and aligned.
template <int TX, int TY>
struct C3Quad {
    using G = C3Tile<TX, TY>;
    static constexpr int NT = G::NT, W = G::W;
    static constexpr int Q1 = G::P1 / 4, Q2 = G::P2 / 4, QO = TX * G::TYO / 4;
    static constexpr int N1 = (Q1 + NT - 1) / NT, N2 = (Q2 + NT - 1) / NT, NO = (QO + NT - 1) / NT;
    static_assert(W % 4 == 0 && TX % 4 == 0, "quads tile the plane rows");
    // u planes are copied ND planes ahead into a ring of ND + 2 slots (one
    // plane deeper than the pair kernels: 2-3% at 512^3); the patch
    // registers hold the ND - 1 pending planes and the current one
    static constexpr int ND = 3, NB = ND + 2;
    static_assert(ND >= 2 && ND <= 3, "three patch register slots");
    static constexpr size_t smem() {
        return (size_t)(NB * G::pua(sizeof(float)) + 3 * G::P1 + 3 * G::P2) * sizeof(float) + NB * 8 + 128;
    }
};

template <int V>
using IC = std::integral_constant<int, V>;

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) chain3d_quad(const C3Args a, const __grid_constant__ CUtensorMap tmap) {
    using G = C3Tile<TX, TY>;
    using Q = C3Quad<TX, TY>;
    constexpr int W = G::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* sbase = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    constexpr int PUS = G::pua(sizeof(float));
    float* U = (float*)sbase;        // [NB][PUS] ring of u planes
    float* S1 = U + Q::NB * PUS;     // [3][P1] ring of s1 planes
    float* S2 = S1 + 3 * G::P1;      // [3][P2] ring of s2 planes
    unsigned long long* bars = (unsigned long long*)(S2 + 3 * G::P2);
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * G::TYO, k0 = blockIdx.z * a.K;
    const float* u = (const float*)a.u.p;
    // periodic edge tiles: the out-of-range band cells of the box, patched
    // from registers loaded two planes ahead (as in chain3d_regw)
    const bool iedge = a.u.wrap && (i0 == 0 || i0 + TX >= a.nx);
    const bool jedge = a.u.wrap && (j0 == 0 || j0 + G::TYO >= a.ny);
    const bool patch = iedge || jedge;
    int pso[G::NF], pgo[G::NF];
    float pv[3][G::NF];
    {
        const int nj = jedge ? 3 : 0, ni = iedge ? 4 : 0;
        const int rj0 = j0 == 0 ? 0 : G::RU - 3;
        const int ci0 = i0 == 0 ? 0 : W - 4;
        const int ro0 = (jedge && j0 == 0) ? 3 : 0;
        const int ncell = nj * W + ni * (G::RU - nj);
#pragma unroll
        for (int f = 0; f < G::NF; ++f) {
            const int e = tid + f * G::NT;
            pso[f] = -1;
            pgo[f] = 0;
            pv[0][f] = pv[1][f] = pv[2][f] = 0.f;
            if (!patch || e >= ncell) continue;
            int r, c;
            if (e < nj * W) { r = rj0 + e / W; c = e % W; }
            else { const int q = e - nj * W; r = ro0 + q / 4; c = ci0 + q % 4; }
            const int gi = wrap_idx(i0 - 4 + c, a.nx), gj = wrap_idx(j0 - 3 + r, a.ny);
            pso[f] = r * W + c;
            pgo[f] = (int)((int64_t)(gj + a.u.org[1]) * a.u.pitch[1] + (gi + a.u.org[0]));
        }
    }
    if (tid == 0) {
        for (int b = 0; b < Q::NB; ++b) mbar_init(bars + b, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // output quads: quad o = tid + r NT is row o / (TX/4), columns 3 + 4 (o % (TX/4)) .. + 3
    float* op[Q::NO];
    int bo[Q::NO];
    bool oko[Q::NO];
#pragma unroll
    for (int r = 0; r < Q::NO; ++r) {
        const int o = tid + r * Q::NT;
        oko[r] = o < Q::QO;
        const int oc = oko[r] ? o : 0;
        const int row = oc / (TX / 4), qc = oc - row * (TX / 4);
        op[r] = garr_ptr<float>(a.out, i0 + 4 * qc, j0 + row, min(k0, a.nz - 1));
        bo[r] = (row + 1) * W + 4 + 4 * qc;
    }
    float4 wu[Q::N1][3], w1[Q::N2][3], w2[Q::NO][3];
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < Q::N1; ++r) wu[r][0] = wu[r][1] = wu[r][2] = zero;
#pragma unroll
    for (int r = 0; r < Q::N2; ++r) w1[r][0] = w1[r][1] = w1[r][2] = zero;
#pragma unroll
    for (int r = 0; r < Q::NO; ++r) w2[r][0] = w2[r][1] = w2[r][2] = zero;
    float wa[7], wb[7];
#pragma unroll
    for (int x = 0; x < 7; ++x) { wa[x] = a.f1[x]; wb[x] = a.f2[x]; }
    const int nu = a.K + 6, nit = a.K + 8;
    const int64_t kstep = a.out.pitch[2];
    bool timed_out = false;
    // u plane it: one tensor copy into slot it % NB; its patch values into pv[D]
    auto fetch = [&](int it, auto D) {
        constexpr int d = decltype(D)::value;
        if (it >= nu) return;
        const int kk = k0 - 3 + it;
        const int kw = a.u.wrap ? wrap1(kk, a.nz) : min(max(kk, -3), a.nz + 2);
        if (tid == 0) {
            unsigned long long* bar = bars + it % Q::NB;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (unsigned)(G::PU * sizeof(float)));
            tma_load_3d(U + (it % Q::NB) * PUS, &tmap, i0 - 4 + a.u.org[0], j0 - 3 + a.u.org[1], kw + a.u.org[2],
                        bar);
        }
        if (patch) {
            const float* pl = u + (int64_t)(kw + a.u.org[2]) * a.u.pitch[2];
#pragma unroll
            for (int f = 0; f < G::NF; ++f)
                if (pso[f] >= 0) pv[d][f] = pl[pgo[f]];
        }
    };
    // one plane iteration; S = it % 3 selects the window slots and rings
    auto step = [&](auto Sc, int it) {
        constexpr int s = decltype(Sc)::value, sp = (s + 1) % 3, sm = (s + 2) % 3;
        if (it < nu) {
            if (!mbar_wait_bounded(bars + it % Q::NB, (unsigned)(it / Q::NB) & 1u, a.err)) timed_out = true;
            if (patch) {
                float* Ub = U + (it % Q::NB) * PUS;
#pragma unroll
                for (int f = 0; f < G::NF; ++f)
                    if (pso[f] >= 0) Ub[pso[f]] = pv[s][f];
            }
        }
        __syncthreads();
        fetch(it + Q::ND, IC<(s + Q::ND) % 3>{});
        // the planes this iteration reads and writes: distinct ring slots, so
        // the stages' shared loads may move ahead of earlier stages' stores
        const float* __restrict__ Ub = U + (it % Q::NB) * PUS;
        const float* __restrict__ Up = U + ((it + Q::NB - 1) % Q::NB) * PUS;
        float* __restrict__ S1b = S1 + s * G::P1;
        const float* __restrict__ S1n = S1 + sm * G::P1;
        const float* __restrict__ S1p = S1 + sp * G::P1;
        float* __restrict__ S2b = S2 + s * G::P2;
        const float* __restrict__ S2n = S2 + sm * G::P2;
        const float* __restrict__ S2p = S2 + sp * G::P2;
        // s1 at plane kk-1 (window slot s holds plane kk, sm kk-1, sp kk-2)
        if (it < nu) {
            const bool comp = it >= 2;
#pragma unroll
            for (int r = 0; r < Q::N1; ++r) {
                const int q = tid + r * Q::NT;
                if (r == Q::N1 - 1 && q >= Q::Q1) continue;
                const int b = 4 * q + W;
                wu[r][s] = *(const float4*)(Ub + b);
                if (!comp) continue;
                const float4 n = *(const float4*)(Up + b + W), so = *(const float4*)(Up + b - W);
                const float l = Up[b - 1], rt = Up[b + 4];
                const float4 c = wu[r][sm], kp = wu[r][s], km = wu[r][sp];
                float4 o;
                o.x = pt7t(wa, c.y, l, n.x, so.x, kp.x, km.x, c.x);
                o.y = pt7t(wa, c.z, c.x, n.y, so.y, kp.y, km.y, c.y);
                o.z = pt7t(wa, c.w, c.y, n.z, so.z, kp.z, km.z, c.z);
                o.w = pt7t(wa, rt, c.z, n.w, so.w, kp.w, km.w, c.w);
                *(float4*)(S1b + 4 * q) = o;
            }
        }
        // s2 at plane kk-3 from the s1 planes made at it-1 (ring slot sm)
        // and it-2 (slot sp)
        if (it >= 3 && it < nu + 1) {
            const bool comp = it >= 5;
#pragma unroll
            for (int r = 0; r < Q::N2; ++r) {
                const int q = tid + r * Q::NT;
                if (r == Q::N2 - 1 && q >= Q::Q2) continue;
                const int b = 4 * q + W;
                w1[r][s] = *(const float4*)(S1n + b);
                if (!comp) continue;
                const float4 n = *(const float4*)(S1p + b + W), so = *(const float4*)(S1p + b - W);
                const float l = S1p[b - 1], rt = S1p[b + 4];
                const float4 c = w1[r][sm], kp = w1[r][s], km = w1[r][sp];
                float4 o;
                o.x = pt7t(wb, c.y, l, n.x, so.x, kp.x, km.x, c.x);
                o.y = pt7t(wb, c.z, c.x, n.y, so.y, kp.y, km.y, c.y);
                o.z = pt7t(wb, c.w, c.y, n.z, so.z, kp.z, km.z, c.z);
                o.w = pt7t(wb, rt, c.z, n.w, so.w, kp.w, km.w, c.w);
                *(float4*)(S2b + 4 * q) = o;
            }
        }
        // out at plane kk-5 from the s2 planes made at it-1 (slot sm) and it-2 (slot sp)
        if (it >= 6) {
            const bool store = it >= 8 && k0 - 8 + it < a.nz;
#pragma unroll
            for (int r = 0; r < Q::NO; ++r) {
                if (!oko[r]) continue;
                const int b = bo[r];
                w2[r][s] = *(const float4*)(S2n + b);
                if (it < 8) continue;
                const float4 n = *(const float4*)(S2p + b + W), so = *(const float4*)(S2p + b - W);
                const float l = S2p[b - 1], rt = S2p[b + 4];
                const float4 c = w2[r][sm], kp = w2[r][s], km = w2[r][sp];
                float4 o;
                o.x = chain3_out<float>(c.y - l, n.x - so.x, kp.x - km.x);
                o.y = chain3_out<float>(c.z - c.x, n.y - so.y, kp.y - km.y);
                o.z = chain3_out<float>(c.w - c.y, n.z - so.z, kp.z - km.z);
                o.w = chain3_out<float>(rt - c.z, n.w - so.w, kp.w - km.w);
                if (store) *(float4*)op[r] = o;
                op[r] += kstep;
            }
        }
    };
    fetch(0, IC<0>{});
    fetch(1, IC<1>{});
    if constexpr (Q::ND == 3) fetch(2, IC<2>{});
    for (int it = 0; it < nit; it += 3) {
        step(IC<0>{}, it);
        if (it + 1 < nit) step(IC<1>{}, it + 1);
        if (it + 2 < nit) step(IC<2>{}, it + 2);
    }
    if (timed_out)
        for (int it = max(0, nu - Q::NB); it < nu; ++it)
            mbar_wait_bounded(bars + it % Q::NB, (unsigned)(it / Q::NB) & 1u, nullptr);
}

namespace {
// planes per CTA for the streaming 3D kernel: with `cap` CTAs resident at a
// time, a launch takes (waves) x (K + lead) iterations; take the K that
// minimises it (ties to the larger K: fewer re-read halo planes)
int chunk_planes(int64_t tiles, int nz, int64_t cap, int lead) {
    int bestK = nz;
    double best = 1e300;
    cap = std::max<int64_t>(cap, 1);
    for (int n = 1; n <= std::min(nz, 1024); ++n) {
        const int K = (nz + n - 1) / n;
        const int64_t ctas = tiles * ((nz + K - 1) / K);
        const double cost = (double)((ctas + cap - 1) / cap) * (K + lead);
        if (cost < best * (1.0 - 1e-9)) { best = cost; bestK = K; }
    }
    return bestK;
}
}  // namespace

// The TMA load form needs the copy 16-byte aligned: the row and plane
// pitches and the column i0 - 4 of a tile (i0 a multiple of TX) after the
// array's halo offset.  On a periodic grid whole tiles (nx a multiple of TX,
// ny of TYO) and at least two per axis, so that a tile patches at most one
// i band and one j band.  Halo-given grids read their halo through the box,
// which starts 4 columns and 3 rows / planes before the interior.
template <typename T, int TX, int TYO>
static bool c3_tma_ok(const C3Args& a) {
    const int A = 16 / (int)sizeof(T);
    const int64_t es = sizeof(T);
    if ((a.u.pitch[1] * es) % 16 || (a.u.pitch[2] * es) % 16 || ((uintptr_t)a.u.p & 15)) return false;
    if (((a.u.org[0] - 4) % A + A) % A) return false;
    if (a.u.wrap) return a.nx % TX == 0 && a.nx >= 2 * TX && a.ny % TYO == 0 && a.ny >= 2 * TYO;
    return a.u.org[0] >= 4 && a.u.org[1] >= 3 && a.u.org[2] >= 3;
}

template <typename T, int TX, int TY, int LOAD>
static int launch_c3regw_load(hfav_plan_t* p, C3Args& a, const CUtensorMap& map, cudaStream_t st) {
    using G = C3Tile<TX, TY>;
    const size_t sm = LOAD == 1 ? G::smem_tma(sizeof(T)) : G::smem(sizeof(T));
    cudaFuncSetAttribute(chain3d_regw<T, TX, TY, LOAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    static int occ = 0;   // resident CTAs per SM (same on every device of the one target)
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chain3d_regw<T, TX, TY, LOAD>, G::NT, sm) !=
                cudaSuccess ||
            occ <= 0) {
            cudaGetLastError();
            occ = 1;
        }
    }
    const int64_t tiles = (int64_t)((a.nx + TX - 1) / TX) * ((a.ny + G::TYO - 1) / G::TYO);
    a.K = chunk_planes(tiles, a.nz, (int64_t)occ * device_sms(), 8);
    dim3 grd((a.nx + TX - 1) / TX, (a.ny + G::TYO - 1) / G::TYO, (a.nz + a.K - 1) / a.K);
    chain3d_regw<T, TX, TY, LOAD><<<grd, dim3(TX, TY), sm, st>>>(a, map);
    HFAV_LAUNCHED(p->rt, LOAD == 1 ? "chain3d_fused_tma" : "chain3d_fused", st);
    return HFAV_OK;
}

template <int TX, int TY>
static int launch_c3quad(hfav_plan_t* p, C3Args& a, const CUtensorMap& map, cudaStream_t st) {
    using G = C3Tile<TX, TY>;
    const size_t sm = C3Quad<TX, TY>::smem();
    cudaFuncSetAttribute(chain3d_quad<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chain3d_quad<TX, TY>, G::NT, sm) != cudaSuccess ||
            occ <= 0) {
            cudaGetLastError();
            occ = 1;
        }
    }
    const int64_t tiles = (int64_t)((a.nx + TX - 1) / TX) * ((a.ny + G::TYO - 1) / G::TYO);
    a.K = chunk_planes(tiles, a.nz, (int64_t)occ * device_sms(), 8);
    dim3 grd((a.nx + TX - 1) / TX, (a.ny + G::TYO - 1) / G::TYO, (a.nz + a.K - 1) / a.K);
    chain3d_quad<TX, TY><<<grd, dim3(TX, TY), sm, st>>>(a, map);
    HFAV_LAUNCHED(p->rt, "chain3d_fused_tma", st);
    return HFAV_OK;
}

template <typename T, int TX, int TY>
static int launch_c3regw(hfav_plan_t* p, C3Args& a, cudaStream_t st) {
    using G = C3Tile<TX, TY>;
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    a.err = (unsigned*)(p->rt->counters + 2);
    if (c3_tma_ok<T, TX, G::TYO>(a)) {
        const int h0 = a.u.org[0], h1 = a.u.org[1], h2 = a.u.org[2];
        const uint64_t dims[3] = {(uint64_t)(a.nx + 2 * h0), (uint64_t)(a.ny + 2 * h1), (uint64_t)(a.nz + 2 * h2)};
        const uint64_t strides[2] = {(uint64_t)(a.u.pitch[1] * sizeof(T)), (uint64_t)(a.u.pitch[2] * sizeof(T))};
        const uint32_t box[3] = {(uint32_t)G::W, (uint32_t)G::RU, 1};
        if (encode_tensor_map_3d(&map, a.u.p, (int)sizeof(T), dims, strides, box)) {
            // quads pay off on the 32-wide tiles (measured at 512^3: 0.495 ms against
            // 0.507 / 0.556 for pairs); the wider tiles keep the pair kernel
            if constexpr (sizeof(T) == 4 && TX == 32) return launch_c3quad<TX, TY>(p, a, map, st);
            else return launch_c3regw_load<T, TX, TY, 1>(p, a, map, st);
        }
    }
    return launch_c3regw_load<T, TX, TY, 0>(p, a, map, st);
}

template <typename T>
static int launch_c3regw_tile(hfav_plan_t* p, const Schedule& s, C3Args& a, cudaStream_t st) {
    if (s.tx == 32 && s.ty == 4) return launch_c3regw<T, 32, 4>(p, a, st);
    if (s.tx == 64 && s.ty == 4) return launch_c3regw<T, 64, 4>(p, a, st);
    if (s.tx == 128 && s.ty == 2) return launch_c3regw<T, 128, 2>(p, a, st);
    if (s.tx == 32 && s.ty == 8) return launch_c3regw<T, 32, 8>(p, a, st);
    return set_error(HFAV_EUNSUPPORTED, "3D chain tile");
}

// tail of the "sweep" schedule: s2 .. out fused from a materialised s1 (halo 2)
template <typename T>
__global__ void __launch_bounds__(256) chain3d_tail(const GArr s1, const GArr out, int nx, int ny, int nz, C3Args a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny || k >= nz) return;
    auto S1 = [&](int x, int y, int z) { return garr_ld<T>(s1, x, y, z); };
    auto S2 = [&](int x, int y, int z) {
        return d7<T>(a.a2, a.f2, S1(x + 1, y, z), S1(x - 1, y, z), S1(x, y + 1, z), S1(x, y - 1, z), S1(x, y, z + 1),
                     S1(x, y, z - 1), S1(x, y, z));
    };
    T gx = S2(i + 1, j, k) - S2(i - 1, j, k), gy = S2(i, j + 1, k) - S2(i, j - 1, k),
      gz = S2(i, j, k + 1) - S2(i, j, k - 1);
    T s3 = sqrt(fma(gx, gx, fma(gy, gy, gz * gz))) * (T)0.5;
    *garr_ptr<T>(out, i, j, k) = s3 / ((T)1 + s3);
}

namespace {
bool star7(const double* w, double* o) {
    // box index (dk+1)*9 + (dj+1)*3 + (di+1)
    static const int idx[7] = {13, 14, 12, 16, 10, 22, 4};
    for (int k = 0; k < 27; ++k) {
        bool star = false;
        for (int m = 0; m < 7; ++m) if (idx[m] == k) star = true;
        if (!star && w[k] != 0.0) return false;
    }
    for (int m = 0; m < 7; ++m) o[m] = w[idx[m]];
    return true;
}
}  // namespace

int launch_chain3d(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st) {
    if (s.fusion == FUSE_UNFUSED) return launch_generic(p, ax, go, st);
    const hfav_grid& g = p->grids[0];
    const ChainMap& m = p->cmap;
    C3Args a;
    memset(&a, 0, sizeof a);
    a.u = caller_view(p, ax[0]);
    a.out = caller_view(p, go[0]);
    a.out.wrap = 0;
    a.nx = (int)g.extent[0]; a.ny = (int)g.extent[1]; a.nz = (int)g.extent[2];
    if (!star7(m.w1, a.a1) || !star7(m.w2, a.a2))
        return set_error(HFAV_EUNSUPPORTED, "fused 3D chain takes 7-point star stencils");
    for (int x = 0; x < 7; ++x) { a.f1[x] = (float)a.a1[x]; a.f2[x] = (float)a.a2[x]; }
    const bool f64 = p->dtype == HFAV_F64;
    const size_t es = esize(p);
    const int TX = s.tx, TY = s.ty;
    if (s.fusion == FUSE_SWEEP) {
        const Rule& R0 = p->dag.rules[m.rules[0]];
        const hfav_field_info& fi = p->an.field[R0.out[0]];
        int64_t e[3];
        for (int x = 0; x < 3; ++x) e[x] = g.extent[x] + fi.halo_lo[x] + fi.halo_hi[x];
        void* ptr;
        int rc = scratch(p, "chain_s1", (size_t)(e[0] * e[1] * e[2]) * es, &ptr);
        if (rc) return rc;
        GArr S;
        S.p = ptr; S.pitch[0] = 1; S.pitch[1] = e[0]; S.pitch[2] = e[0] * e[1];
        for (int x = 0; x < 3; ++x) { S.org[x] = fi.halo_lo[x]; S.ext[x] = (int)g.extent[x]; }
        S.wrap = 0;
        GenericArgs ga;
        memset(&ga, 0, sizeof ga);
        ga.op = HFAV_OP_STENCIL_LINEAR;
        ga.nref = (int)R0.in.size();
        ga.arr[0] = a.u;
        for (int k = 0; k < ga.nref; ++k) {
            for (int x = 0; x < 3; ++x) ga.ref_off[k][x] = R0.in[k].off[x];
            ga.w[k] = R0.params[k];
        }
        ga.out = S;
        for (int x = 0; x < 3; ++x) { ga.lo[x] = -fi.halo_lo[x]; ga.n[x] = (int)e[x]; }
        int64_t tot = e[0] * e[1] * e[2];
        int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)device_sms() * 16);
        for (int k = 0; k < 27; ++k) ga.wf[k] = (float)ga.w[k];
        if (f64) generic_rule_kernel<double><<<blocks, 256, 0, st>>>(ga);
        else generic_rule_kernel<float><<<blocks, 256, 0, st>>>(ga);
        HFAV_LAUNCHED(p->rt, "generic_rule_kernel", st);
        dim3 blk(TX, TY), grd((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, a.nz);
        if (f64) chain3d_tail<double><<<grd, blk, 0, st>>>(S, a.out, a.nx, a.ny, a.nz, a);
        else chain3d_tail<float><<<grd, blk, 0, st>>>(S, a.out, a.nx, a.ny, a.nz, a);
        HFAV_LAUNCHED(p->rt, "chain3d_tail", st);
        return HFAV_OK;
    }
    if (s.placement == PLACE_REG)
        return f64 ? launch_c3regw_tile<double>(p, s, a, st) : launch_c3regw_tile<float>(p, s, a, st);
    // chunk of planes per CTA: enough CTAs to fill the machine
    int64_t tiles = (int64_t)((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY);
    int K = 8;
    while (K < 64 && tiles * ((a.nz + 2 * K - 1) / (2 * K)) >= (int64_t)device_sms() * 8) K *= 2;
    a.K = K;
    dim3 blk(TX, TY), grd((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + K - 1) / K);
    size_t per = (size_t)3 * ((TX + 6) * (TY + 6) + (TX + 4) * (TY + 4) + (TX + 2) * (TY + 2)) * es;
    if (s.placement == PLACE_HBM) {
        void* slab;
        int rc = scratch(p, "chain3d_slab", per * grd.x * grd.y * grd.z, &slab);
        if (rc) return rc;
        a.slab = slab;
        if (f64) chain3d_ring<double, true><<<grd, blk, 0, st>>>(a);
        else chain3d_ring<float, true><<<grd, blk, 0, st>>>(a);
    } else {
        if (per > 200 * 1024) return set_error(HFAV_EUNSUPPORTED, "3D tile too large for shared memory");
        if (f64) {
            cudaFuncSetAttribute(chain3d_ring<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)per);
            chain3d_ring<double, false><<<grd, blk, per, st>>>(a);
        } else {
            cudaFuncSetAttribute(chain3d_ring<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)per);
            chain3d_ring<float, false><<<grd, blk, per, st>>>(a);
        }
    }
    HFAV_LAUNCHED(p->rt, "chain3d_fused", st);
    return HFAV_OK;
}

}  // namespace hfav

// ---------------------------------------------------------------------------
// resident warps per SM of the chain kernel a schedule launches (its main
// kernel), for the schedule model's features; -1 without a usable device
// ---------------------------------------------------------------------------
namespace hfav {
namespace {
template <typename K>
double warps_of(K kern, int threads, size_t smem) {
    int occ = 0;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    return (double)occ * threads / 32.0;
}
template <typename T>
double chain_warps_t(const hfav_plan_t* p, const Schedule& s) {
    const int TX = s.tx, TY = s.ty, NT = TX * TY;
    const size_t es = sizeof(T);
    if (s.fusion == FUSE_UNFUSED) return warps_of(generic_rule_kernel<T>, 256, 0);
    if (p->pipeline == PIPE_CHAIN2D) {
        if (s.fusion == FUSE_SWEEP) return warps_of(chain2d_tail<T>, NT, 0);
        if (s.placement == PLACE_REG)
            return c2w_wide(TX, TY) ? warps_of(chain2d_warp<T, 16 / sizeof(T)>, NT, 0)
                                    : warps_of(chain2d_warp<T, 8 / sizeof(T)>, NT, 0);
        if (s.placement == PLACE_SMEM)
            return warps_of(chain2d_ring<T, false>, NT, (size_t)TY * (3 * (TX + 4) + 3 * (TX + 2)) * es);
        return warps_of(chain2d_ring<T, true>, NT, 0);
    }
    if (s.fusion == FUSE_SWEEP) return warps_of(chain3d_tail<T>, NT, 0);
    if (s.placement == PLACE_REG) {
#define C3W(a, b)                                                                                             \
    if (TX == a && TY == b) {                                                                                 \
        using G = C3Tile<a, b>;                                                                               \
        if constexpr (sizeof(T) == 4 && a == 32) return warps_of(chain3d_quad<a, b>, NT, C3Quad<a, b>::smem());   \
        return warps_of(chain3d_regw<T, a, b, 1>, NT, G::smem_tma(es));                                       \
    }
        C3W(32, 4) C3W(64, 4) C3W(128, 2) C3W(32, 8)
#undef C3W
        return -1.0;
    }
    const size_t per = (size_t)3 * ((TX + 6) * (TY + 6) + (TX + 4) * (TY + 4) + (TX + 2) * (TY + 2)) * es;
    if (s.placement == PLACE_SMEM) return warps_of(chain3d_ring<T, false>, NT, per);
    return warps_of(chain3d_ring<T, true>, NT, 0);
}
}  // namespace

double chain_kernel_warps(const hfav_plan_t* p, const Schedule& s) {
    return p->dtype == HFAV_F64 ? chain_warps_t<double>(p, s) : chain_warps_t<float>(p, s);
}
}  // namespace hfav
