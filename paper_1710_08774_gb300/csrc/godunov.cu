// godunov.cu -- the directionally split 2D Euler Godunov step (Hydro2D's nine
// kernels, HFAV Sec. 5.4) as fused GPU pipelines, plus the unfused form.
//
// Schedules (fusion axis of the plan):
//   sweep   -- the paper's fusion: all nine kernels of one pass in one nest
//              (Sec. 5.4 "fuse all nine ... into a single loop nest"), one
//              kernel per pass: gsweep_x then gsweep_y.  The CFL reduction of
//              the next step is fused into gsweep_y's epilogue.
//   full    -- both passes in one kernel (gfull): every CTA x-sweeps the rows
//              of its strip into a shared row and streams them through a
//              5-row (skewed: 3-row) y window; it recomputes the x-sweep on a
//              2-row / 1-column halo.
//   unfused -- every kernel its own launch over fully materialised arrays.
// Placement (where the y windows live between rows): reg | smem | hbm.
// The x pass always stages its row in shared memory (neighbour exchange along
// the contiguous axis), or in a per-CTA global slab for placement hbm.
//
// Work lists: every fused kernel walks a list of (grid, item) pairs, so one
// launch covers a whole batch of grids of different sizes; a single grid is a
// batch of one.  The time step of grid g at step s is dt = cfl dx / wave[s]
// with wave[s] the max wave speed of the state entering step s (bits of a
// non-negative double, reduced with atomicMax); dt/dx = cfl / wave[s].
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "godunov_phys.cuh"

namespace hfav {

template <typename T>
struct GGrid {
    const T* src[4];
    T* dst[4];
    int64_t spitch, dpitch;
    int shalo, dhalo;
    int nx, ny;
    unsigned long long* wave;   // wave[step] read, wave[step + 1] reduced into
    int xS, xseg, xfull;        // x pass: segment length, segments per row, full periodic row
    int yR, ystrips, ychunks;   // y pass: rows per thread, column strips, row chunks
};

struct GCommon {
    double cfl, gamma;
    double ig1;            // 1 / (gamma - 1)
    double ashk;           // (gamma + 1) / (2 gamma), the shock coefficient of the Riemann solver
    float gammaf, ig1f;    // gamma and 1 / (gamma - 1) rounded to FP32 on the host, so an
                           // FP32 kernel converts no FP64 parameter on the device
    int step;
    unsigned long long* counters;   // [0] Newton non-converged faces, [1] non-physical cells
    void* slab;                     // per-CTA-group scratch for placement hbm
    int reduce_cfl;                 // gsweep_y / gfull: fold the next step's CFL reduction in
    int newton_max;                 // cap on the Riemann solver's Newton iterations
};

template <typename T>
__device__ __forceinline__ T csel(double d, float f) {
    if constexpr (sizeof(T) == 8) return (T)d;
    else return (T)f;
}

template <typename T>
__device__ __forceinline__ T ldg_src(const GGrid<T>& G, int f, int i, int j) {
    return G.src[f][(int64_t)(j + G.shalo) * G.spitch + (i + G.shalo)];
}

template <typename T>
__device__ __forceinline__ void st_dst(const GGrid<T>& G, int f, int i, int j, T v) {
    G.dst[f][(int64_t)(j + G.dhalo) * G.dpitch + (i + G.dhalo)] = v;
}

__device__ __forceinline__ double dtdx_of(const GGrid<float>& G, int step, double cfl) {
    return cfl / __longlong_as_double((long long)G.wave[step]);
}
__device__ __forceinline__ double dtdx_of(const GGrid<double>& G, int step, double cfl) {
    return cfl / __longlong_as_double((long long)G.wave[step]);
}

// primitive state rebuilt from the five staged values (r, un, ut, p, s),
// s = rsqrt(g p r): c = g p s, 1/c = r s, c/r = c^2 s
template <typename T>
__device__ __forceinline__ Prim<T> prim5(T r, T un, T ut, T p, T s, T g) {
    Prim<T> w;
    w.r = r; w.un = un; w.ut = ut; w.p = p;
    w.c = g * p * s;
    w.ic = r * s;
    w.cr = w.c * w.c * s;
    return w;
}

template <typename T>
__device__ __forceinline__ void cfl_epilogue(double smax, int bad, int nonconv, const GCommon& C,
                                             unsigned long long* wave_next) {
    smax = warp_max(smax);
    unsigned any_nc = __ballot_sync(0xffffffffu, nonconv);
    unsigned any_bad = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (C.reduce_cfl && smax > 0.0) atomic_max_pos(wave_next, smax);
        if (any_nc) atomicAdd(&C.counters[0], (unsigned long long)__popc(any_nc));
        if (any_bad) atomicAdd(&C.counters[1], (unsigned long long)__popc(any_bad));
    }
}

// ---------------------------------------------------------------------------
// x pass, placement reg: one warp per row streams along i in chunks of 32
// cells with the rolling buffers in registers and neighbours exchanged by
// warp shuffles -- the GPU form of the paper's vector-widened rotation of an
// innermost-dimension buffer (Sec. 3.5 "Vectorization").  Chunk v covers
// cells 32 v - 1 + lane.  Step s computes W of chunk s, the trace of chunk
// s-1 and the faces (right face of each cell) and updates of chunk s-2.
// Rows with nx % 32 == 0 are exact-periodic: nx faces, nx traces, and one
// extra W chunk per row; other rows run a halo form (nx+1 faces).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ Prim<T> shfl_prim(const Prim<T>& w, int src) {
    Prim<T> o;
    o.r = __shfl_sync(0xffffffffu, w.r, src); o.un = __shfl_sync(0xffffffffu, w.un, src);
    o.ut = __shfl_sync(0xffffffffu, w.ut, src); o.p = __shfl_sync(0xffffffffu, w.p, src);
    o.c = __shfl_sync(0xffffffffu, w.c, src); o.ic = __shfl_sync(0xffffffffu, w.ic, src);
    o.cr = __shfl_sync(0xffffffffu, w.cr, src);
    return o;
}
template <typename T>
__device__ __forceinline__ Face4<T> shfl_face(const Face4<T>& q, int src) {
    Face4<T> o;
    o.r = __shfl_sync(0xffffffffu, q.r, src); o.u = __shfl_sync(0xffffffffu, q.u, src);
    o.v = __shfl_sync(0xffffffffu, q.v, src); o.p = __shfl_sync(0xffffffffu, q.p, src);
    return o;
}

template <typename T>
__global__ void __launch_bounds__(256, 2) gsweep_xw(const GGrid<T>* __restrict__ grids, const int2* __restrict__ items,
                                                 int n_items, const GCommon C) {
    // one CTA per row; its A warps split the row into A arcs of equal length
    // (rows with nx % (32 A) != 0 use one arc).  Arc w streams the faces of
    // cells a0-1 .. a0+La-2; the face of its last cell is the first face of
    // arc w+1 and the qm of that face's right state is arc w+1's first trace:
    // both cross through shared memory.
    __shared__ Face4<T> s_qm[8], s_F[8];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int A = blockDim.x >> 5;
    const T g = csel<T>(C.gamma, C.gammaf), ig1 = csel<T>(C.ig1, C.ig1f);
    const double ashk = C.ashk;
    int nonconv = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const GGrid<T>& G = grids[it.x];
        const int j = it.y, nx = G.nx;
        const bool exact = (nx & 31) == 0;
        const int arcs = (exact && nx % (32 * A) == 0) ? A : 1;
        const bool active = w < arcs;
        const int La = exact ? nx / arcs : nx;
        const int a0 = active ? w * La : 0;
        const int nf = exact ? La : nx + 1;           // faces of cells a0-1 .. a0+nf-2
        const int nch = (nf + 31) >> 5;
        const T dtdx = (T)dtdx_of(G, C.step, C.cfl);
        auto load_prim = [&](int i) {
            const int iw = wrap_idx(i, nx);
            return cons_to_prim(ldg_src(G, 0, iw, j), ldg_src(G, 1, iw, j), ldg_src(G, 2, iw, j), ldg_src(G, 3, iw, j), g);
        };
        Prim<T> Wold, carryW;
        if (active) {
            Wold = load_prim(a0 - 33 + lane);          // chunk -1 (only lane 31, cell a0-2, is used)
            carryW = shfl_prim(Wold, 31);
            Wold = load_prim(a0 - 1 + lane);           // chunk 0
        }
        Face4<T> qmOld, qpOld, qmNext, Fsave, carryF;
        for (int s = 1; s <= nch + 1; ++s) {
            const bool wstep = !(exact && s == nch + 1);
            Prim<T> Wcur = Wold;
            Face4<T> qmNew, qpNew;
            if (active && wstep) {
                Wcur = load_prim(a0 + 32 * s - 1 + lane);
                Prim<T> wl = shfl_prim(Wold, (lane + 31) & 31);
                if (lane == 0) wl = carryW;
                Prim<T> wr = shfl_prim(Wold, (lane + 1) & 31);
                Prim<T> w0n = shfl_prim(Wcur, 0);
                if (lane == 31) wr = w0n;
                slope_trace(wl, Wold, wr, dtdx, qmNew, qpNew);   // cells of chunk s-1
                carryW = shfl_prim(Wold, 31);
                if (s == 1 && exact) {
                    Face4<T> q0 = shfl_face(qmNew, 0);   // qm of cell a0-1
                    if (lane == 0) s_qm[w] = q0;
                }
            }
            if (s == 1) {
                __syncthreads();
                if (active && exact) qmNext = s_qm[(w + 1) % arcs];   // qm of cell a0+La-1
            }
            if (active && s >= 2) {
                const int v = s - 2;
                const int cell = a0 + 32 * v - 1 + lane;
                Face4<T> qR = shfl_face(qmOld, (lane + 1) & 31);
                Face4<T> q0n = (exact && s == nch + 1) ? qmNext : shfl_face(qmNew, 0);
                if (lane == 31) qR = q0n;
                int nc_local = 0;
                Face4<T> F = flux(riemann(qpOld, qR, g, ashk, C.newton_max, &nc_local), ig1);
                if (32 * v - 1 + lane <= nf - 2) nonconv |= nc_local;
                if (v == 0) {
                    Fsave = shfl_face(F, 0);   // face of cell a0-1
                    if (lane == 0) s_F[w] = Fsave;
                }
                Face4<T> Fl = shfl_face(F, (lane + 31) & 31);
                if (lane == 0) Fl = carryF;
                carryF = shfl_face(F, 31);
                // update with left face Fl and right face F (cell a0-1 belongs
                // to the previous arc; in exact form the arc's last cell waits
                // for the next arc's first face)
                const bool upd = (32 * v - 1 + lane >= 0) && cell < (exact ? a0 + La - 1 : nx) && cell >= 0;
                if (upd) {
                    st_dst(G, 0, cell, j, fma(-dtdx, F.r - Fl.r, ldg_src(G, 0, cell, j)));
                    st_dst(G, 1, cell, j, fma(-dtdx, F.u - Fl.u, ldg_src(G, 1, cell, j)));
                    st_dst(G, 2, cell, j, fma(-dtdx, F.v - Fl.v, ldg_src(G, 2, cell, j)));
                    st_dst(G, 3, cell, j, fma(-dtdx, F.p - Fl.p, ldg_src(G, 3, cell, j)));
                }
            }
            qmOld = qmNew; qpOld = qpNew;
            Wold = Wcur;
        }
        __syncthreads();
        // exact form: the last cell of the arc, between the arc's last face
        // (carryF) and the next arc's first face
        if (active && exact && lane == 0) {
            const Face4<T> Fr = s_F[(w + 1) % arcs];
            const int cell = a0 + La - 1;
            st_dst(G, 0, cell, j, fma(-dtdx, Fr.r - carryF.r, ldg_src(G, 0, cell, j)));
            st_dst(G, 1, cell, j, fma(-dtdx, Fr.u - carryF.u, ldg_src(G, 1, cell, j)));
            st_dst(G, 2, cell, j, fma(-dtdx, Fr.v - carryF.v, ldg_src(G, 2, cell, j)));
            st_dst(G, 3, cell, j, fma(-dtdx, Fr.p - carryF.p, ldg_src(G, 3, cell, j)));
        }
        __syncthreads();
    }
    unsigned any_nc = __ballot_sync(0xffffffffu, nonconv);
    if (lane == 0 && any_nc) atomicAdd(&C.counters[0], (unsigned long long)__popc(any_nc));
}

// ---------------------------------------------------------------------------
// x pass, placement smem / hbm: one row (or row segment) per CTA, staged in
// shared memory or in a per-CTA global slab.  Staging (elements of T):
// W 5 x (S+4) [r un ut p s], qm 4 x (S+2), qp 4 x (S+2); fluxes 4 x (S+1)
// reuse the W area.  A segment of S cells needs W on [-2, S+2), traces on
// [-1, S], faces [0, S]; a full periodic row (S == nx) needs W, traces and
// faces on [0, S) only.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t xstage_elems(int S) {
    return (size_t)5 * (S + 4) + (size_t)8 * (S + 2);
}

template <typename T, bool HBM>
__global__ void __launch_bounds__(256) gsweep_x(const GGrid<T>* __restrict__ grids, const int2* __restrict__ items,
                                                int n_items, int Smax, const GCommon C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NT = blockDim.x * blockDim.y, t = threadIdx.y * blockDim.x + threadIdx.x;
    const size_t per = xstage_elems<T>(Smax);
    T* st;
    if (HBM) st = (T*)C.slab + (size_t)blockIdx.x * per;
    else st = (T*)smem_raw;
    const T g = csel<T>(C.gamma, C.gammaf), ig1 = csel<T>(C.ig1, C.ig1f);
    const double ashk = C.ashk;
    int nonconv = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const GGrid<T>& G = grids[it.x];
        const int S = G.xS, full = G.xfull;
        const int j = it.y / G.xseg, seg = it.y % G.xseg;
        const int s0 = seg * S;
        const int WS = S + 4, QS = S + 2;
        T* W = st;                 // [5][WS], index l + 2
        T* QM = st + 5 * WS;       // [4][QS], index l + 1
        T* QP = QM + 4 * QS;       // [4][QS], index l + 1
        T* F = st;                 // [4][S+1] after the traces
        const T dtdx = (T)dtdx_of(G, C.step, C.cfl);
        {
            const int lo = full ? 0 : -2, hi = full ? S : S + 2;
            for (int l = lo + t; l < hi; l += NT) {
                int i = wrap_idx(s0 + l, G.nx);
                Prim<T> w = cons_to_prim(ldg_src(G, 0, i, j), ldg_src(G, 1, i, j), ldg_src(G, 2, i, j), ldg_src(G, 3, i, j), g);
                W[0 * WS + l + 2] = w.r; W[1 * WS + l + 2] = w.un; W[2 * WS + l + 2] = w.ut;
                W[3 * WS + l + 2] = w.p; W[4 * WS + l + 2] = w.ic / w.r;
            }
        }
        __syncthreads();
        {
            const int lo = full ? 0 : -1, hi = full ? S : S + 1;
            for (int l = lo + t; l < hi; l += NT) {
                int lm = l - 1, lp = l + 1;
                if (full) { lm = lm < 0 ? lm + S : lm; lp = lp >= S ? lp - S : lp; }
                Prim<T> wm = prim5(W[lm + 2], W[WS + lm + 2], W[2 * WS + lm + 2], W[3 * WS + lm + 2], W[4 * WS + lm + 2], g);
                Prim<T> w0 = prim5(W[l + 2], W[WS + l + 2], W[2 * WS + l + 2], W[3 * WS + l + 2], W[4 * WS + l + 2], g);
                Prim<T> wp = prim5(W[lp + 2], W[WS + lp + 2], W[2 * WS + lp + 2], W[3 * WS + lp + 2], W[4 * WS + lp + 2], g);
                Face4<T> qm, qp;
                slope_trace(wm, w0, wp, dtdx, qm, qp);
                QM[0 * QS + l + 1] = qm.r; QM[1 * QS + l + 1] = qm.u; QM[2 * QS + l + 1] = qm.v; QM[3 * QS + l + 1] = qm.p;
                QP[0 * QS + l + 1] = qp.r; QP[1 * QS + l + 1] = qp.u; QP[2 * QS + l + 1] = qp.v; QP[3 * QS + l + 1] = qp.p;
            }
        }
        __syncthreads();
        {
            const int nf = full ? S : S + 1;
            for (int l = t; l < nf; l += NT) {
                int lm = l - 1;
                if (full && lm < 0) lm += S;
                Face4<T> L, R;
                L.r = QP[lm + 1]; L.u = QP[QS + lm + 1]; L.v = QP[2 * QS + lm + 1]; L.p = QP[3 * QS + lm + 1];
                R.r = QM[l + 1]; R.u = QM[QS + l + 1]; R.v = QM[2 * QS + l + 1]; R.p = QM[3 * QS + l + 1];
                Face4<T> fl = flux(riemann(L, R, g, ashk, C.newton_max, &nonconv), ig1);
                F[0 * (S + 1) + l] = fl.r; F[1 * (S + 1) + l] = fl.u; F[2 * (S + 1) + l] = fl.v; F[3 * (S + 1) + l] = fl.p;
            }
        }
        __syncthreads();
        for (int l = t; l < S; l += NT) {
            int i = s0 + l;
            if (i >= G.nx) break;
            int lp = l + 1;
            if (full && lp == S) lp = 0;
            T f0 = F[lp] - F[l], f1 = F[(S + 1) + lp] - F[(S + 1) + l];
            T f2 = F[2 * (S + 1) + lp] - F[2 * (S + 1) + l], f3 = F[3 * (S + 1) + lp] - F[3 * (S + 1) + l];
            st_dst(G, 0, i, j, fma(-dtdx, f0, ldg_src(G, 0, i, j)));
            st_dst(G, 1, i, j, fma(-dtdx, f1, ldg_src(G, 1, i, j)));
            st_dst(G, 2, i, j, fma(-dtdx, f2, ldg_src(G, 2, i, j)));
            st_dst(G, 3, i, j, fma(-dtdx, f3, ldg_src(G, 3, i, j)));
        }
        __syncthreads();
    }
    unsigned any_nc = __ballot_sync(0xffffffffu, nonconv);
    if ((t & 31) == 0 && any_nc) atomicAdd(&C.counters[0], (unsigned long long)__popc(any_nc));
}

// ---------------------------------------------------------------------------
// y pass: one thread per column streams a chunk of rows.  Windows (skewed
// pipeline): W of rows r-2, r-1, r; U of rows r-2, r-1; qp of row r-2; flux
// of the face below row r-1.  Placement: registers, or a per-thread ring in
// shared memory / a global slab that the window makes a round trip through
// every row.
// ---------------------------------------------------------------------------
template <typename T>
struct YWin {
    Prim<T> W0, W1;
    Face4<T> U0, U1, qpp, Fp;
};

// number of T values of one thread's window ring
#define YWIN_VALS 38

template <typename T>
__device__ __forceinline__ void ywin_store(volatile T* p, int stride, const YWin<T>& w) {
    const T v[YWIN_VALS] = {w.W0.r, w.W0.un, w.W0.ut, w.W0.p, w.W0.c, w.W0.ic, w.W0.cr,
                            w.W1.r, w.W1.un, w.W1.ut, w.W1.p, w.W1.c, w.W1.ic, w.W1.cr,
                            w.U0.r, w.U0.u, w.U0.v, w.U0.p, w.U1.r, w.U1.u, w.U1.v, w.U1.p,
                            w.qpp.r, w.qpp.u, w.qpp.v, w.qpp.p, w.Fp.r, w.Fp.u, w.Fp.v, w.Fp.p,
                            0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 30; ++k) p[k * stride] = v[k];
}

template <typename T>
__device__ __forceinline__ void ywin_load(const volatile T* p, int stride, YWin<T>& w) {
    T v[30];
#pragma unroll
    for (int k = 0; k < 30; ++k) v[k] = p[k * stride];
    w.W0 = Prim<T>{v[0], v[1], v[2], v[3], v[4], v[5], v[6]};
    w.W1 = Prim<T>{v[7], v[8], v[9], v[10], v[11], v[12], v[13]};
    w.U0 = Face4<T>{v[14], v[15], v[16], v[17]};
    w.U1 = Face4<T>{v[18], v[19], v[20], v[21]};
    w.qpp = Face4<T>{v[22], v[23], v[24], v[25]};
    w.Fp = Face4<T>{v[26], v[27], v[28], v[29]};
}

// One row of the y pipeline for a thread: U2 is the conserved state of row r
// in the y frame (rho, rho v, rho u, E).  Emits the updated cell r-2 into out.
template <typename T>
__device__ __forceinline__ bool ystep(YWin<T>& w, const Face4<T>& U2, int r, int j0, T dtdx, T g, double ashk, T ig1,
                                      int nmax, int* nonconv, Face4<T>* out) {
    Prim<T> W2 = cons_to_prim(U2.r, U2.u, U2.v, U2.p, g);
    bool emit = false;
    if (r >= j0) {
        Face4<T> qm, qp;
        slope_trace(w.W0, w.W1, W2, dtdx, qm, qp);   // cell r-1
        if (r >= j0 + 1) {
            Face4<T> q = riemann(w.qpp, qm, g, ashk, nmax, nonconv);   // face between r-2 and r-1
            Face4<T> F = flux(q, ig1);
            if (r >= j0 + 2) {   // update cell r-2 with its faces below (Fp) and above (F)
                out->r = fma(-dtdx, F.r - w.Fp.r, w.U0.r);
                out->u = fma(-dtdx, F.u - w.Fp.u, w.U0.u);
                out->v = fma(-dtdx, F.v - w.Fp.v, w.U0.v);
                out->p = fma(-dtdx, F.p - w.Fp.p, w.U0.p);
                emit = true;
            }
            w.Fp = F;
        }
        w.qpp = qp;
    }
    w.W0 = w.W1; w.W1 = W2;
    w.U0 = w.U1; w.U1 = U2;
    return emit;
}

template <typename T, int PL>
__global__ void __launch_bounds__(256, PL == PLACE_REG ? 2 : 1) gsweep_y(const GGrid<T>* __restrict__ grids, const int2* __restrict__ items,
                                                int n_items, const GCommon C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = blockDim.x, t = threadIdx.x, ty = threadIdx.y, TY = blockDim.y;
    const T g = csel<T>(C.gamma, C.gammaf), ig1 = csel<T>(C.ig1, C.ig1f);
    const double ashk = C.ashk;
    const int lane_slot = ty * TX + t;
    volatile T* ring = nullptr;
    int stride = 0;
    if (PL == PLACE_SMEM) { ring = (volatile T*)smem_raw + lane_slot; stride = TX * TY; }
    if (PL == PLACE_HBM) {
        ring = (volatile T*)C.slab + (size_t)blockIdx.x * TX * TY * YWIN_VALS + lane_slot;
        stride = TX * TY;
    }
    int nonconv = 0, bad = 0;
    for (int base = blockIdx.x * TY; base < n_items; base += gridDim.x * TY) {
        const int item = base + ty;
        double smax = 0.0;
        unsigned long long* wave_next = nullptr;
        if (item < n_items) {
            const int2 it = items[item];
            const GGrid<T>& G = grids[it.x];
            wave_next = G.wave + C.step + 1;
            const int strip = it.y % G.ystrips, chunk = it.y / G.ystrips;
            const int i = strip * TX + t;
            const int j0 = chunk * G.yR;
            if (i < G.nx) {
                const T dtdx = (T)dtdx_of(G, C.step, C.cfl);
                YWin<T> w;
                memset(&w, 0, sizeof w);
                for (int r = j0 - 2; r <= j0 + G.yR + 1; ++r) {
                    const int jr = wrap_idx(r, G.ny);
                    Face4<T> U2;
                    U2.r = ldg_src(G, 0, i, jr); U2.u = ldg_src(G, 2, i, jr);
                    U2.v = ldg_src(G, 1, i, jr); U2.p = ldg_src(G, 3, i, jr);
                    if (PL != PLACE_REG && r > j0 - 2) ywin_load(ring, stride, w);
                    Face4<T> o;
                    bool emit = ystep(w, U2, r, j0, dtdx, g, ashk, ig1, C.newton_max, &nonconv, &o);
                    if (PL != PLACE_REG) ywin_store(ring, stride, w);
                    const int j = r - 2;
                    if (emit && j < G.ny) {
                        st_dst(G, 0, i, j, o.r); st_dst(G, 2, i, j, o.u);
                        st_dst(G, 1, i, j, o.v); st_dst(G, 3, i, j, o.p);
                        smax = speed_max(smax, wave_speed(o.r, o.v, o.u, o.p, g, &bad));
                    }
                }
            }
        }
        // all lanes of a warp share the item (TX is a multiple of 32)
        if (item < n_items) cfl_epilogue<T>(smax, bad, nonconv, C, wave_next);
        nonconv = 0; bad = 0;
    }
}

// ---------------------------------------------------------------------------
// full step in one kernel: a group of TX threads owns a strip of TX-2
// columns and a chunk of R rows.  For every row r of [j0-2, j0+R+1] the group
// x-sweeps cells [-2, TX) of the strip (W), traces [-1, TX-2], solves faces
// [0, TX-2] and updates [0, TX-3] into a shared row; then thread t streams
// column t of that row through the y pipeline.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline size_t fstage_elems(int TX) {
    return (size_t)5 * (TX + 2) + (size_t)8 * TX + (size_t)4 * TX;
}

template <typename T, int PL>
__global__ void __launch_bounds__(256) gfull(const GGrid<T>* __restrict__ grids, const int2* __restrict__ items,
                                             int n_items, const GCommon C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = blockDim.x, t = threadIdx.x, ty = threadIdx.y, TY = blockDim.y;
    const T g = csel<T>(C.gamma, C.gammaf), ig1 = csel<T>(C.ig1, C.ig1f);
    const double ashk = C.ashk;
    const size_t per = fstage_elems<T>(TX);
    T* st = (T*)smem_raw + ty * per;
    const int WS = TX + 2;
    T* Wst = st;              // [5][TX+2], cell c at c + 2
    T* QM = st + 5 * WS;      // [4][TX], cell c at c + 1
    T* QP = QM + 4 * TX;      // [4][TX]
    T* UR = QP + 4 * TX;      // [4][TX]  x-updated row
    T* F = st;                // [4][TX]  fluxes after the traces
    volatile T* ring = nullptr;
    int stride = 0;
    const int lane_slot = ty * TX + t;
    T* rings_base = (T*)smem_raw + TY * per;
    if (PL == PLACE_SMEM) { ring = (volatile T*)rings_base + lane_slot; stride = TX * TY; }
    if (PL == PLACE_HBM) {
        ring = (volatile T*)C.slab + (size_t)blockIdx.x * TX * TY * YWIN_VALS + lane_slot;
        stride = TX * TY;
    }
    int nonconv = 0, bad = 0;
    for (int base = blockIdx.x * TY; base < n_items; base += gridDim.x * TY) {
        const int item = base + ty;
        const bool active = item < n_items;
        const int2 it = active ? items[item] : make_int2(0, 0);
        const GGrid<T>& G = grids[it.x];
        const int strip = it.y % G.ystrips, chunk = it.y / G.ystrips;
        const int i0 = strip * (TX - 2), j0 = chunk * G.yR;
        const T dtdx = active ? (T)dtdx_of(G, C.step, C.cfl) : (T)0;
        double smax = 0.0;
        YWin<T> w;
        memset(&w, 0, sizeof w);
        const int R = active ? G.yR : 0;
        // every group of the CTA runs the same number of rows (barriers)
        int Rmax = R;
        for (int k = 0; k < TY; ++k) {
            int itk = base + k;
            if (itk < n_items) Rmax = max(Rmax, grids[items[itk].x].yR);
        }
        for (int r = j0 - 2; r <= j0 + Rmax + 1; ++r) {
            const bool row_on = active && r <= j0 + R + 1;
            const int jr = row_on ? wrap_idx(r, G.ny) : 0;
            // W on cells c in [-2, TX): thread t takes c = t - 2 and (t < 2) c = TX - 2 + t
            if (row_on) {
                for (int c = t - 2; c < TX; c += TX) {
                    int i = wrap_idx(i0 + c, G.nx);
                    Prim<T> pw = cons_to_prim(ldg_src(G, 0, i, jr), ldg_src(G, 1, i, jr), ldg_src(G, 2, i, jr),
                                              ldg_src(G, 3, i, jr), g);
                    Wst[c + 2] = pw.r; Wst[WS + c + 2] = pw.un; Wst[2 * WS + c + 2] = pw.ut;
                    Wst[3 * WS + c + 2] = pw.p; Wst[4 * WS + c + 2] = pw.ic / pw.r;
                    if (t >= 2) break;
                }
            }
            __syncthreads();
            // traces of cells c = t - 1 in [-1, TX-2]
            if (row_on) {
                const int c = t - 1;
                Prim<T> wm = prim5(Wst[c + 1], Wst[WS + c + 1], Wst[2 * WS + c + 1], Wst[3 * WS + c + 1], Wst[4 * WS + c + 1], g);
                Prim<T> w0 = prim5(Wst[c + 2], Wst[WS + c + 2], Wst[2 * WS + c + 2], Wst[3 * WS + c + 2], Wst[4 * WS + c + 2], g);
                Prim<T> wp = prim5(Wst[c + 3], Wst[WS + c + 3], Wst[2 * WS + c + 3], Wst[3 * WS + c + 3], Wst[4 * WS + c + 3], g);
                Face4<T> qm, qp;
                slope_trace(wm, w0, wp, dtdx, qm, qp);
                QM[c + 1] = qm.r; QM[TX + c + 1] = qm.u; QM[2 * TX + c + 1] = qm.v; QM[3 * TX + c + 1] = qm.p;
                QP[c + 1] = qp.r; QP[TX + c + 1] = qp.u; QP[2 * TX + c + 1] = qp.v; QP[3 * TX + c + 1] = qp.p;
            }
            __syncthreads();
            // faces l = t in [0, TX-2]: left face of cell l
            if (row_on && t <= TX - 2) {
                const int l = t;
                Face4<T> L, Rr;
                L.r = QP[l]; L.u = QP[TX + l]; L.v = QP[2 * TX + l]; L.p = QP[3 * TX + l];
                Rr.r = QM[l + 1]; Rr.u = QM[TX + l + 1]; Rr.v = QM[2 * TX + l + 1]; Rr.p = QM[3 * TX + l + 1];
                Face4<T> fl = flux(riemann(L, Rr, g, ashk, C.newton_max, &nonconv), ig1);
                F[l] = fl.r; F[TX + l] = fl.u; F[2 * TX + l] = fl.v; F[3 * TX + l] = fl.p;
            }
            __syncthreads();
            // x update of cells c = t in [0, TX-3] into the shared row
            if (row_on && t <= TX - 3) {
                const int i = wrap_idx(i0 + t, G.nx);
                UR[t] = fma(-dtdx, F[t + 1] - F[t], ldg_src(G, 0, i, jr));
                UR[TX + t] = fma(-dtdx, F[TX + t + 1] - F[TX + t], ldg_src(G, 1, i, jr));
                UR[2 * TX + t] = fma(-dtdx, F[2 * TX + t + 1] - F[2 * TX + t], ldg_src(G, 2, i, jr));
                UR[3 * TX + t] = fma(-dtdx, F[3 * TX + t + 1] - F[3 * TX + t], ldg_src(G, 3, i, jr));
            }
            __syncthreads();
            // y pipeline of column t
            if (row_on && t <= TX - 3 && i0 + t < G.nx) {
                Face4<T> U2;
                U2.r = UR[t]; U2.u = UR[2 * TX + t]; U2.v = UR[TX + t]; U2.p = UR[3 * TX + t];
                if (PL != PLACE_REG && r > j0 - 2) ywin_load(ring, stride, w);
                Face4<T> o;
                bool emit = ystep(w, U2, r, j0, dtdx, g, ashk, ig1, C.newton_max, &nonconv, &o);
                if (PL != PLACE_REG) ywin_store(ring, stride, w);
                const int j = r - 2;
                if (emit && j < G.ny) {
                    const int i = i0 + t;
                    st_dst(G, 0, i, j, o.r); st_dst(G, 2, i, j, o.u);
                    st_dst(G, 1, i, j, o.v); st_dst(G, 3, i, j, o.p);
                    smax = speed_max(smax, wave_speed(o.r, o.v, o.u, o.p, g, &bad));
                }
            }
        }
        if (active) cfl_epilogue<T>(smax, bad, nonconv, C, G.wave + C.step + 1);
        nonconv = 0; bad = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// CFL reduction of a state (the first step of a run, and every step of the
// unfused form): wave[slot] = max over cells of max(|u|+c, |v|+c)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) gcfl_reduce(const GGrid<T>* __restrict__ grids, int n_grids, int slot,
                                                   double gamma, unsigned long long* counters, int use_dst) {
    const int gi = blockIdx.y;
    if (gi >= n_grids) return;
    const GGrid<T>& G = grids[gi];
    const int64_t n = (int64_t)G.nx * G.ny;
    double smax = 0.0;
    int bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(k % G.nx), j = (int)(k / G.nx);
        T u[4];
        for (int f = 0; f < 4; ++f)
            u[f] = use_dst ? G.dst[f][(int64_t)(j + G.dhalo) * G.dpitch + i + G.dhalo] : ldg_src(G, f, i, j);
        smax = speed_max(smax, wave_speed(u[0], u[1], u[2], u[3], (T)gamma, &bad));
    }
    smax = warp_max(smax);
    const unsigned any_bad = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(G.wave + slot, smax);
        if (any_bad) atomicAdd(&counters[1], (unsigned long long)__popc(any_bad));
    }
}

// ---------------------------------------------------------------------------
// unfused form: every Hydro2D kernel its own launch over materialised arrays
// (plan-owned, padded by 2 cells, pitch P).  Face a+1/2 is stored at a.
// ---------------------------------------------------------------------------
template <typename T>
struct UArrays {
    T *U[4], *r, *un, *ut, *e, *p, *c, *dW[4], *qm[4], *qp[4], *qL[4], *qR[4], *gd[4], *F[4];
    int64_t P;
    int nx, ny;
};

template <typename T>
__device__ __forceinline__ int64_t uidx(const UArrays<T>& A, int dir, int a, int b) {
    int i = dir == 0 ? a : b, j = dir == 0 ? b : a;
    return (int64_t)(j + 2) * A.P + (i + 2);
}

#define U_LOOP(lo_a, hi_a)                                                                              \
    const int na = dir == 0 ? A.nx : A.ny, nb = dir == 0 ? A.ny : A.nx;                                 \
    const int64_t span = (int64_t)((hi_a) - (lo_a));                                                    \
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < span * nb;                     \
         k += (int64_t)gridDim.x * blockDim.x) {                                                        \
        const int a = (int)(k % span) + (lo_a), b = (int)(k / span);                                    \
        (void)na;

template <typename T>
__global__ void u_make_boundary(const GGrid<T> G, UArrays<T> A) {
    const int64_t n = (int64_t)(A.nx + 4) * (A.ny + 4);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(k % (A.nx + 4)) - 2, j = (int)(k / (A.nx + 4)) - 2;
        int si = wrap_idx(i, A.nx), sj = wrap_idx(j, A.ny);
        for (int f = 0; f < 4; ++f) A.U[f][(int64_t)(j + 2) * A.P + (i + 2)] = ldg_src(G, f, si, sj);
    }
}

template <typename T>
__global__ void u_constoprim(UArrays<T> A, int dir) {
    U_LOOP(-2, na + 2)
        const int64_t x = uidx(A, dir, a, b);
        const int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
        T r = A.U[0][x];
        T ir = (T)1 / r;
        T un = A.U[mn][x] * ir, ut = A.U[mt][x] * ir;
        A.r[x] = r; A.un[x] = un; A.ut[x] = ut;
        A.e[x] = fma(A.U[3][x], ir, -dhalf(fma(un, un, ut * ut)));
    }
}

template <typename T>
__global__ void u_eos(UArrays<T> A, int dir, T g) {
    U_LOOP(-2, na + 2)
        const int64_t x = uidx(A, dir, a, b);
        T r = A.r[x];
        if (r < (T)G_RHO_FLOOR) { r = (T)G_RHO_FLOOR; A.r[x] = r; }
        T p = (g - (T)1) * r * A.e[x];
        p = p > (T)G_P_FLOOR ? p : (T)G_P_FLOOR;
        A.p[x] = p;
        A.c[x] = sqrt(g * p / r);
    }
}

template <typename T>
__global__ void u_slope(UArrays<T> A, int dir) {
    U_LOOP(-1, na + 1)
        const int64_t x = uidx(A, dir, a, b), xm = uidx(A, dir, a - 1, b), xp = uidx(A, dir, a + 1, b);
        const T* q[4] = {A.r, A.un, A.ut, A.p};
        for (int f = 0; f < 4; ++f) A.dW[f][x] = minmod(q[f][x] - q[f][xm], q[f][xp] - q[f][x]);
    }
}

template <typename T>
__global__ void u_trace(UArrays<T> A, int dir, const GGrid<T>* G, int step, double cfl) {
    const T dtdx = (T)dtdx_of(*G, step, cfl);
    U_LOOP(-1, na + 1)
        const int64_t x = uidx(A, dir, a, b);
        Prim<T> w;
        w.r = A.r[x]; w.un = A.un[x]; w.ut = A.ut[x]; w.p = A.p[x]; w.c = A.c[x];
        w.ic = (T)1 / w.c;
        w.cr = w.c / w.r;
        Face4<T> qm, qp;
        trace(w, A.dW[0][x], A.dW[1][x], A.dW[2][x], A.dW[3][x], dtdx, qm, qp);
        A.qm[0][x] = qm.r; A.qm[1][x] = qm.u; A.qm[2][x] = qm.v; A.qm[3][x] = qm.p;
        A.qp[0][x] = qp.r; A.qp[1][x] = qp.u; A.qp[2][x] = qp.v; A.qp[3][x] = qp.p;
    }
}

template <typename T>
__global__ void u_qleftright(UArrays<T> A, int dir) {
    U_LOOP(-1, na)
        const int64_t x = uidx(A, dir, a, b), xp = uidx(A, dir, a + 1, b);
        for (int f = 0; f < 4; ++f) { A.qL[f][x] = A.qp[f][x]; A.qR[f][x] = A.qm[f][xp]; }
    }
}

template <typename T>
__global__ void u_riemann(UArrays<T> A, int dir, T g, double ashk, int nmax, unsigned long long* counters) {
    int nonconv = 0;
    U_LOOP(-1, na)
        const int64_t x = uidx(A, dir, a, b);
        Face4<T> L{A.qL[0][x], A.qL[1][x], A.qL[2][x], A.qL[3][x]};
        Face4<T> R{A.qR[0][x], A.qR[1][x], A.qR[2][x], A.qR[3][x]};
        Face4<T> q = riemann(L, R, g, ashk, nmax, &nonconv);
        A.gd[0][x] = q.r; A.gd[1][x] = q.u; A.gd[2][x] = q.v; A.gd[3][x] = q.p;
    }
    unsigned m = __ballot_sync(0xffffffffu, nonconv);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&counters[0], (unsigned long long)__popc(m));
}

template <typename T>
__global__ void u_cmpflx(UArrays<T> A, int dir, T ig1) {
    U_LOOP(-1, na)
        const int64_t x = uidx(A, dir, a, b);
        Face4<T> q{A.gd[0][x], A.gd[1][x], A.gd[2][x], A.gd[3][x]};
        Face4<T> F = flux(q, ig1);
        A.F[0][x] = F.r; A.F[1][x] = F.u; A.F[2][x] = F.v; A.F[3][x] = F.p;
    }
}

template <typename T>
__global__ void u_update(UArrays<T> A, int dir, const GGrid<T>* G, int step, double cfl) {
    const T dtdx = (T)dtdx_of(*G, step, cfl);
    U_LOOP(0, na)
        const int64_t x = uidx(A, dir, a, b), xm = uidx(A, dir, a - 1, b);
        const int mn = dir == 0 ? 1 : 2, mt = dir == 0 ? 2 : 1;
        const int i = dir == 0 ? a : b, j = dir == 0 ? b : a;
        st_dst(*G, 0, i, j, fma(-dtdx, A.F[0][x] - A.F[0][xm], A.U[0][x]));
        st_dst(*G, mn, i, j, fma(-dtdx, A.F[1][x] - A.F[1][xm], A.U[mn][x]));
        st_dst(*G, mt, i, j, fma(-dtdx, A.F[2][x] - A.F[2][xm], A.U[mt][x]));
        st_dst(*G, 3, i, j, fma(-dtdx, A.F[3][x] - A.F[3][xm], A.U[3][x]));
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct GodState {
    // per grid device pointers of the plan-owned state buffers
    std::vector<std::array<void*, 4>> P, X;   // ping-pong state, x-swept state
    std::vector<int64_t> pitch;               // pitch of plan-owned state arrays (halo 0)
};

int64_t round_up(int64_t a, int64_t m) { return (a + m - 1) / m * m; }

template <typename T>
struct Tables {
    GGrid<T>* dev = nullptr;   // [kinds][n_grids]
    int2* xitems = nullptr;
    int2* yitems = nullptr;
    int nx_items = 0, ny_items = 0;
    int Smax = 0;
};

// state kinds: 0 axioms, 1 goals, 2 plan ping-pong, 3 x-swept scratch
template <typename T>
int state_ptrs(hfav_plan_t* p, int kind, int g, void* const* ax, void* const* go, T** out, int64_t* pitch,
               int* halo) {
    const hfav_grid& G = p->grids[g];
    if (kind == 0 || kind == 1) {
        void* const* src = kind == 0 ? ax : go;
        for (int f = 0; f < 4; ++f) out[f] = (T*)src[g * 4 + f];
        *pitch = G.pitch[1];
        *halo = G.halo;
        return HFAV_OK;
    }
    const int64_t P = round_up(G.extent[0], 32);
    const size_t bytes = (size_t)P * G.extent[1] * sizeof(T);
    for (int f = 0; f < 4; ++f) {
        void* ptr;
        int rc = scratch(p, std::string(kind == 2 ? "gstate_" : "gxswept_") + std::to_string(g) + "_" + std::to_string(f),
                         bytes, &ptr);
        if (rc) return rc;
        out[f] = (T*)ptr;
    }
    *pitch = P;
    *halo = 0;
    return HFAV_OK;
}

// grid decomposition (x segments, y strips / chunks) for one schedule
template <typename T>
void decompose(const hfav_plan_t* p, const Schedule& s, int g, GGrid<T>& G, int Smax, int yR) {
    const hfav_grid& H = p->grids[g];
    const int nx = (int)H.extent[0], ny = (int)H.extent[1];
    G.nx = nx; G.ny = ny;
    // staged x pass: a full periodic row when it fits the staging and fills
    // whole warps, else segments of k*32-2 cells (k*32-1 faces, k*32 traces)
    if (nx <= Smax && nx % 32 == 0) { G.xS = nx; G.xseg = 1; G.xfull = 1; }
    else {
        int kmax = (Smax + 2) / 32;
        int nseg = (nx + kmax * 32 - 3) / (kmax * 32 - 2);
        int k = (nx / nseg + 2 + 31) / 32;
        while ((k * 32 - 2) * nseg < nx) ++k;
        G.xS = k * 32 - 2; G.xseg = nseg; G.xfull = 0;
    }
    const int W = s.fusion == FUSE_FULL ? s.tx - 2 : s.tx;
    int R = std::min(yR, std::max(4, ny));
    G.yR = R;
    G.ystrips = (nx + W - 1) / W;
    G.ychunks = (ny + R - 1) / R;
}

// Rows per y item.  A y item is TX/32 warps streaming R rows (plus a 4-row
// prologue whose faces, traces and states are recomputed).  On a part whose
// FP64 pipe is the bottleneck the pass ends when the busiest SM sub-partition
// (608 of them) has drained its warps, so R is chosen to minimise
// ceil(warps / 608) * (R + 1.5), with a penalty when fewer than two warps per
// sub-partition are left to hide latency.
int choose_yR(const hfav_plan_t* p, const Schedule& s) {
    const int W = s.fusion == FUSE_FULL ? s.tx - 2 : s.tx;
    const int wpi = s.tx / 32;
    double best = 1e30;
    int bestR = 16;
    for (int R = 8; R <= 256; ++R) {
        int64_t warps = 0;
        for (auto& g : p->grids)
            warps += (int64_t)((g.extent[0] + W - 1) / W) * ((g.extent[1] + R - 1) / R) * wpi;
        const int64_t slots = (int64_t)device_sms() * 4;
        const int64_t q = (warps + slots - 1) / slots;
        const double cost = q * (R + 1.5) / (q >= 2 ? 1.0 : 0.6);
        if (cost < best - 1e-9) { best = cost; bestR = R; }
    }
    return bestR;
}

// largest staged x segment whose staging stays within ~100 KB (two CTAs per SM)
int smax_for(const hfav_plan_t* p, size_t es) {
    int maxnx = 0;
    for (auto& g : p->grids) maxnx = std::max<int>(maxnx, (int)g.extent[0]);
    const size_t budget = 100 * 1024;
    int S = 30;
    while ((size_t)(5 * (S + 32 + 4) + 8 * (S + 32 + 2)) * es <= budget && S + 32 <= 4094) S += 32;
    if (maxnx % 32 == 0 && maxnx > S && (size_t)(5 * (maxnx + 4) + 8 * (maxnx + 2)) * es <= budget) S = maxnx;
    return std::max(S, std::min(maxnx, S));
}

}  // namespace

template <typename T>
static int run_godunov_t(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, int n_steps,
                         cudaStream_t st) {
    Runtime* rt = p->rt;
    const int ng = (int)p->grids.size();
    const size_t es = sizeof(T);
    const GodunovMap& gm = p->gmap;
    const int Smax = smax_for(p, es);
    const int yR = choose_yR(p, s);
    // wave slots: n_steps + 1 per grid
    if (rt->wave_cap < n_steps + 1 || !rt->wave) {
        int cap = std::max(n_steps + 1, 128);
        void* w;
        int rc = scratch(p, "wave", (size_t)cap * ng * sizeof(unsigned long long), &w);
        if (rc) return rc;
        rt->wave = (unsigned long long*)w;
        rt->wave_cap = cap;
    }
    HFAV_CUDA(cudaMemsetAsync(rt->wave, 0, (size_t)rt->wave_cap * ng * sizeof(unsigned long long), st));
    HFAV_CUDA(cudaMemsetAsync(rt->counters, 0, 2 * sizeof(unsigned long long), st));

    // host tables for the (src, dst) kinds used by this run; kinds per step:
    // step s reads state(s) and writes state(s+1); state(0) = axioms,
    // state(n) = goals, between them the goals / plan buffer alternate so the
    // last write lands in the goals and the axioms are never written.
    auto state_kind = [&](int k) {
        if (k == 0) return 0;
        return ((n_steps - k) % 2 == 0) ? 1 : 2;
    };
    std::vector<GGrid<T>> host;   // tables back to back
    std::map<std::pair<int, int>, int> tix;
    auto table = [&](int sk, int dk) -> int {
        auto key = std::make_pair(sk, dk);
        auto itt = tix.find(key);
        if (itt != tix.end()) return itt->second;
        int at = (int)host.size();
        for (int g = 0; g < ng; ++g) {
            GGrid<T> G;
            memset(&G, 0, sizeof G);
            T* sp[4]; T* dp[4];
            int64_t spitch, dpitch;
            int shalo, dhalo;
            if (state_ptrs<T>(p, sk, g, ax, go, sp, &spitch, &shalo)) return -1;
            if (state_ptrs<T>(p, dk, g, ax, go, dp, &dpitch, &dhalo)) return -1;
            for (int f = 0; f < 4; ++f) { G.src[f] = sp[f]; G.dst[f] = dp[f]; }
            G.spitch = spitch; G.dpitch = dpitch; G.shalo = shalo; G.dhalo = dhalo;
            G.wave = rt->wave + (size_t)g * rt->wave_cap;
            decompose<T>(p, s, g, G, Smax, yR);
            host.push_back(G);
        }
        tix[key] = at;
        return at;
    };
    struct StepTabs { int x, y, full, cfl0; };
    std::vector<StepTabs> steps(n_steps);
    for (int k = 0; k < n_steps; ++k) {
        int sk = state_kind(k), dk = state_kind(k + 1);
        if (s.fusion == FUSE_SWEEP) { steps[k].x = table(sk, 3); steps[k].y = table(3, dk); }
        else { steps[k].full = table(sk, dk); steps[k].x = table(sk, 3); steps[k].y = table(3, dk); }
        if (steps[k].x < 0 || steps[k].y < 0) return set_error(HFAV_ENOMEM, "state buffers");
    }
    int t0 = table(0, 3);
    if (t0 < 0) return set_error(HFAV_ENOMEM, "state buffers");
    // work items
    std::vector<int2> xit, yit;
    {
        const GGrid<T>* G0 = &host[t0];
        for (int g = 0; g < ng; ++g)
            for (int k = 0; k < G0[g].ny * G0[g].xseg; ++k) xit.push_back(make_int2(g, k));
        for (int g = 0; g < ng; ++g)
            for (int k = 0; k < G0[g].ystrips * G0[g].ychunks; ++k) yit.push_back(make_int2(g, k));
        // heavier grids first so the persistent CTAs end together
        std::stable_sort(xit.begin(), xit.end(), [&](int2 a, int2 b) { return G0[a.x].nx > G0[b.x].nx; });
        std::stable_sort(yit.begin(), yit.end(), [&](int2 a, int2 b) { return G0[a.x].yR > G0[b.x].yR; });
    }
    // the tables hold this run's pointers: uploaded in stream order, so a
    // run queued behind an earlier one never changes the tables under it
    void *dtab, *dxit, *dyit;
    int rc;
    if ((rc = upload(p, "gtables", host.data(), host.size() * sizeof(GGrid<T>), st, &dtab))) return rc;
    if ((rc = upload(p, "gxitems", xit.data(), xit.size() * sizeof(int2), st, &dxit))) return rc;
    if ((rc = upload(p, "gyitems", yit.data(), yit.size() * sizeof(int2), st, &dyit))) return rc;
    const GGrid<T>* tabs = (const GGrid<T>*)dtab;

    GCommon C;
    C.cfl = gm.cfl;
    C.gamma = gm.gamma;
    C.ig1 = 1.0 / (gm.gamma - 1.0);
    C.ashk = 0.5 * (gm.gamma + 1.0) / gm.gamma;
    C.gammaf = (float)C.gamma;
    C.ig1f = (float)C.ig1;
    C.counters = rt->counters;
    C.slab = nullptr;
    C.reduce_cfl = 1;
    C.newton_max = gm.newton_max;

    const int TX = s.tx, TY = s.ty;
    // step 0's wave speed
    {
        dim3 grd(std::max(1, std::min(64, (int)(xit.size() / 4 + 1))), ng);
        gcfl_reduce<T><<<grd, 256, 0, st>>>(tabs + t0, ng, 0, gm.gamma, rt->counters, 0);
        HFAV_LAUNCHED(rt, "gcfl_reduce", st);
    }
    if (s.fusion == FUSE_UNFUSED) {
        if (ng != 1) return set_error(HFAV_EUNSUPPORTED, "unfused form runs one grid");
        const hfav_grid& H = p->grids[0];
        UArrays<T> A;
        A.nx = (int)H.extent[0]; A.ny = (int)H.extent[1];
        A.P = round_up(A.nx + 4, 32);
        const size_t bytes = (size_t)A.P * (A.ny + 4) * es;
        T** slots[] = {&A.U[0], &A.U[1], &A.U[2], &A.U[3], &A.r, &A.un, &A.ut, &A.e, &A.p, &A.c,
                       &A.dW[0], &A.dW[1], &A.dW[2], &A.dW[3], &A.qm[0], &A.qm[1], &A.qm[2], &A.qm[3],
                       &A.qp[0], &A.qp[1], &A.qp[2], &A.qp[3], &A.qL[0], &A.qL[1], &A.qL[2], &A.qL[3],
                       &A.qR[0], &A.qR[1], &A.qR[2], &A.qR[3], &A.gd[0], &A.gd[1], &A.gd[2], &A.gd[3],
                       &A.F[0], &A.F[1], &A.F[2], &A.F[3]};
        int k = 0;
        for (T** sl : slots) {
            void* ptr;
            if ((rc = scratch(p, "unf_" + std::to_string(k++), bytes, &ptr))) return rc;
            *sl = (T*)ptr;
        }
        const int64_t cells = (int64_t)(A.nx + 4) * (A.ny + 4);
        const int blocks = (int)std::min<int64_t>((cells + 255) / 256, (int64_t)device_sms() * 16);
        const T g = (T)gm.gamma, ig1 = (T)(1.0 / (gm.gamma - 1.0));
        for (int step = 0; step < n_steps; ++step) {
            const GGrid<T>* tx_ = tabs + steps[step].x;   // state(step) -> x-swept
            const GGrid<T>* ty_ = tabs + steps[step].y;   // x-swept -> state(step+1)
            if (step > 0) {   // CFL as its own nest over the state entering the step
                gcfl_reduce<T><<<dim3(64, 1), 256, 0, st>>>(tx_, 1, step, gm.gamma, rt->counters, 0);
                HFAV_LAUNCHED(rt, "gcfl_reduce", st);
            }
            for (int dir = 0; dir < 2; ++dir) {
                const GGrid<T>* G = dir == 0 ? tx_ : ty_;
                GGrid<T> Gh = host[dir == 0 ? steps[step].x : steps[step].y];
                u_make_boundary<T><<<blocks, 256, 0, st>>>(Gh, A); HFAV_LAUNCHED(rt, "u_make_boundary", st);
                u_constoprim<T><<<blocks, 256, 0, st>>>(A, dir); HFAV_LAUNCHED(rt, "u_constoprim", st);
                u_eos<T><<<blocks, 256, 0, st>>>(A, dir, g); HFAV_LAUNCHED(rt, "u_eos", st);
                u_slope<T><<<blocks, 256, 0, st>>>(A, dir); HFAV_LAUNCHED(rt, "u_slope", st);
                u_trace<T><<<blocks, 256, 0, st>>>(A, dir, G, step, gm.cfl); HFAV_LAUNCHED(rt, "u_trace", st);
                u_qleftright<T><<<blocks, 256, 0, st>>>(A, dir); HFAV_LAUNCHED(rt, "u_qleftright", st);
                u_riemann<T><<<blocks, 256, 0, st>>>(A, dir, g, C.ashk, C.newton_max, rt->counters); HFAV_LAUNCHED(rt, "u_riemann", st);
                u_cmpflx<T><<<blocks, 256, 0, st>>>(A, dir, ig1); HFAV_LAUNCHED(rt, "u_cmpflx", st);
                u_update<T><<<blocks, 256, 0, st>>>(A, dir, G, step, gm.cfl); HFAV_LAUNCHED(rt, "u_update", st);
            }
        }
        // the wave speed of the final state (for the dt history / status)
        gcfl_reduce<T><<<dim3(64, 1), 256, 0, st>>>(tabs + steps[n_steps - 1].y, 1, n_steps, gm.gamma,
                                                   rt->counters, 1);
        HFAV_LAUNCHED(rt, "gcfl_reduce", st);
        return HFAV_OK;
    }
    // persistent grids: the SMs times the resident CTAs of each kernel
    const int kSMs = device_sms();
    if (s.fusion == FUSE_SWEEP) {
        const int NT = TX * TY;
        const size_t xsm = xstage_elems<T>(Smax) * es;
        const size_t ysm = s.placement == PLACE_SMEM ? (size_t)NT * YWIN_VALS * es : 0;
        int occx = 1, occy = 1;
        // x pass work: rows (warp-streaming form) or row segments (staged form)
        std::vector<int2> xrows;
        for (int g = 0; g < ng; ++g)
            for (int k = 0; k < (int)p->grids[g].extent[1]; ++k) xrows.push_back(make_int2(g, k));
        std::stable_sort(xrows.begin(), xrows.end(), [&](int2 a, int2 b) {
            return p->grids[a.x].extent[0] > p->grids[b.x].extent[0];
        });
        void* dxrows = nullptr;
        // arcs per row: the most arcs (warps per row) for which every row is
        // resident at once -- a row is the unit of work, so a second partial
        // wave leaves SMs idle -- and at least two warps per SM sub-partition
        int xarcs = 1;
        {
            const int64_t rows = (int64_t)xrows.size();
            int minnx = 1 << 30;
            for (auto& q : p->grids) minnx = std::min<int>(minnx, (int)q.extent[0]);
            cudaFuncAttributes fa;
            int regs = 128;
            if (cudaFuncGetAttributes(&fa, gsweep_xw<T>) == cudaSuccess) regs = std::max(fa.numRegs, 1);
            else cudaGetLastError();
            for (int A = 8; A >= 1; A /= 2) {
                if (minnx < 32 * 2 * A) continue;   // at least two chunks per arc
                const int64_t per_sm = std::min<int64_t>(65536 / (32 * A * regs), 2048 / (32 * A));
                if (rows <= per_sm * kSMs && rows * A >= (int64_t)kSMs * 4 * 2) { xarcs = A; break; }
            }
            if (xarcs == 1) {   // rows exceed one wave: enough arcs for ~6 warps per sub-partition
                while (xarcs < 8 && rows * xarcs < (int64_t)kSMs * 4 * 6 && minnx >= 32 * 2 * xarcs * 2) xarcs *= 2;
            }
        }
        if (s.placement == PLACE_REG) {
            if ((rc = upload(p, "gxrows", xrows.data(), xrows.size() * sizeof(int2), st, &dxrows))) return rc;
            HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occx, gsweep_xw<T>, 32 * xarcs, 0));
        } else if (s.placement == PLACE_HBM) {
            HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occx, gsweep_x<T, true>, NT, 0));
        } else {
            HFAV_CUDA(cudaFuncSetAttribute(gsweep_x<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm));
            HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occx, gsweep_x<T, false>, NT, xsm));
        }
        auto ykern = s.placement == PLACE_REG ? gsweep_y<T, PLACE_REG>
                     : s.placement == PLACE_SMEM ? gsweep_y<T, PLACE_SMEM> : gsweep_y<T, PLACE_HBM>;
        if (ysm > 48 * 1024) HFAV_CUDA(cudaFuncSetAttribute(ykern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm));
        HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occy, ykern, NT, ysm));
        occx = std::max(occx, 1); occy = std::max(occy, 1);
        int gx;
        if (s.placement == PLACE_REG)
            gx = (int)std::min<int64_t>((int64_t)xrows.size(), (int64_t)kSMs * occx);
        else
            gx = (int)std::min<int64_t>((int64_t)xit.size(), (int64_t)kSMs * occx);
        int gy = (int)std::min<int64_t>(((int64_t)yit.size() + TY - 1) / TY, (int64_t)kSMs * occy);
        if (s.placement == PLACE_HBM) {
            size_t need = std::max((size_t)gx * xstage_elems<T>(Smax), (size_t)gy * NT * YWIN_VALS) * es;
            if ((rc = scratch(p, "gslab", need, &C.slab))) return rc;
        }
        for (int step = 0; step < n_steps; ++step) {
            C.step = step;
            if (s.placement == PLACE_REG)
                gsweep_xw<T><<<gx, 32 * xarcs, 0, st>>>(tabs + steps[step].x, (const int2*)dxrows, (int)xrows.size(), C);
            else if (s.placement == PLACE_HBM)
                gsweep_x<T, true><<<gx, NT, 0, st>>>(tabs + steps[step].x, (const int2*)dxit, (int)xit.size(), Smax, C);
            else
                gsweep_x<T, false><<<gx, NT, xsm, st>>>(tabs + steps[step].x, (const int2*)dxit, (int)xit.size(), Smax, C);
            HFAV_LAUNCHED(rt, "gsweep_x", st);
            ykern<<<gy, dim3(TX, TY), ysm, st>>>(tabs + steps[step].y, (const int2*)dyit, (int)yit.size(), C);
            HFAV_LAUNCHED(rt, "gsweep_y", st);
        }
        return HFAV_OK;
    }
    // full fusion: items are (strip of TX-2 columns, chunk) -- the y items of
    // a decomposition with strip width TX-2
    {
        const size_t fsm = (size_t)TY * fstage_elems<T>(TX) * es +
                           (s.placement == PLACE_SMEM ? (size_t)TX * TY * YWIN_VALS * es : 0);
        auto fk = s.placement == PLACE_REG ? gfull<T, PLACE_REG>
                  : s.placement == PLACE_SMEM ? gfull<T, PLACE_SMEM> : gfull<T, PLACE_HBM>;
        HFAV_CUDA(cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
        int occ = 1;
        HFAV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk, TX * TY, fsm));
        occ = std::max(occ, 1);
        int gf = (int)std::min<int64_t>(((int64_t)yit.size() + TY - 1) / TY, (int64_t)kSMs * occ);
        if (s.placement == PLACE_HBM) {
            if ((rc = scratch(p, "gslab", (size_t)gf * TX * TY * YWIN_VALS * es, &C.slab))) return rc;
        }
        for (int step = 0; step < n_steps; ++step) {
            C.step = step;
            fk<<<gf, dim3(TX, TY), fsm, st>>>(tabs + steps[step].full, (const int2*)dyit, (int)yit.size(), C);
            HFAV_LAUNCHED(rt, "gfull", st);
        }
    }
    return HFAV_OK;
}

int launch_godunov(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, int n_steps,
                   cudaStream_t st) {
    if (p->dtype == HFAV_F64) return run_godunov_t<double>(p, s, ax, go, n_steps, st);
    return run_godunov_t<float>(p, s, ax, go, n_steps, st);
}

}  // namespace hfav

// ---------------------------------------------------------------------------
// diagnostic: the Newton-refined reciprocal and quotient of the kernels on an
// array, so tests can hold them against IEEE division
// ---------------------------------------------------------------------------
namespace hfav {
__global__ void selftest_arith_k(const double* __restrict__ x, int64_t n, double* __restrict__ r,
                                 double* __restrict__ q) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        r[k] = rcp_nr(x[k]);
        q[k] = div_nr(1.5, x[k]);
    }
}
__global__ void selftest_rsqrt_k(const double* __restrict__ x, int64_t n, double* __restrict__ r) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        r[k] = newton_rsqrt<float>(x[k]);
}
__global__ void selftest_half_k(const double* __restrict__ x, int64_t n, double* __restrict__ r) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        r[k] = dhalf(x[k]);
}
__global__ void selftest_convert_k(const double* __restrict__ x, const float* __restrict__ f, int64_t n,
                                   float* __restrict__ nr, double* __restrict__ wd) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        nr[k] = narrow(x[k]);
        wd[k] = widen(f[k]);
    }
}
}  // namespace hfav

extern "C" int hfav_selftest_convert(const double* x, const float* f, int64_t n, float* narrow_out, double* widen_out,
                                     void* stream) {
    using namespace hfav;
    if (!x || !f || !narrow_out || !widen_out || n < 0) return set_error(HFAV_EINVAL, "bad argument");
    if (n == 0) return HFAV_OK;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    selftest_convert_k<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, f, n, narrow_out, widen_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, cudaGetErrorString(e));
    return HFAV_OK;
}

extern "C" int hfav_selftest_half(const double* x, int64_t n, double* out, void* stream) {
    using namespace hfav;
    if (!x || !out || n < 0) return set_error(HFAV_EINVAL, "bad argument");
    if (n == 0) return HFAV_OK;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    selftest_half_k<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, n, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, cudaGetErrorString(e));
    return HFAV_OK;
}

extern "C" int hfav_selftest_rsqrt(const double* x, int64_t n, double* out, void* stream) {
    using namespace hfav;
    if (!x || !out || n < 0) return set_error(HFAV_EINVAL, "bad argument");
    if (n == 0) return HFAV_OK;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    selftest_rsqrt_k<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, n, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, cudaGetErrorString(e));
    return HFAV_OK;
}

extern "C" int hfav_selftest_arith(const double* x, int64_t n, double* rcp_out, double* quot_out, void* stream) {
    using namespace hfav;
    if (!x || !rcp_out || !quot_out || n < 0) return set_error(HFAV_EINVAL, "bad argument");
    if (n == 0) return HFAV_OK;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    selftest_arith_k<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, n, rcp_out, quot_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, cudaGetErrorString(e));
    return HFAV_OK;
}

namespace hfav {
namespace {
template <typename K>
double gwarps_of(K kern, int threads, size_t smem) {
    int occ = 0;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    return (double)occ * threads / 32.0;
}
template <typename T>
double godunov_warps_t(const Schedule& s) {
    const int NT = s.tx * s.ty;
    const size_t es = sizeof(T);
    if (s.fusion == FUSE_UNFUSED) return gwarps_of(u_riemann<T>, 256, 0);
    if (s.fusion == FUSE_SWEEP) {   // the y pass takes the larger share
        const size_t ysm = s.placement == PLACE_SMEM ? (size_t)NT * YWIN_VALS * es : 0;
        if (s.placement == PLACE_REG) return gwarps_of(gsweep_y<T, PLACE_REG>, NT, 0);
        if (s.placement == PLACE_SMEM) return gwarps_of(gsweep_y<T, PLACE_SMEM>, NT, ysm);
        return gwarps_of(gsweep_y<T, PLACE_HBM>, NT, 0);
    }
    const size_t fsm = (size_t)s.ty * fstage_elems<T>(s.tx) * es +
                       (s.placement == PLACE_SMEM ? (size_t)NT * YWIN_VALS * es : 0);
    if (s.placement == PLACE_REG) return gwarps_of(gfull<T, PLACE_REG>, NT, fsm);
    if (s.placement == PLACE_SMEM) return gwarps_of(gfull<T, PLACE_SMEM>, NT, fsm);
    return gwarps_of(gfull<T, PLACE_HBM>, NT, fsm);
}
}  // namespace

double godunov_kernel_warps(const hfav_plan_t* p, const Schedule& s) {
    return p->dtype == HFAV_F64 ? godunov_warps_t<double>(s) : godunov_warps_t<float>(s);
}
}  // namespace hfav
