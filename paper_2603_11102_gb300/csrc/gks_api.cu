// gks_api.cu -- host side of the C ABI declared in include/gks_api.h: grid
// validation, carving of the caller-owned buffers, geometry tables, object
// set-up, and the launch sequence of one S2O4 step.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gks_internal.h"

using namespace gks;

struct Profiler {
    bool timing = false;
    bool nvtx = false;   // NVTX range per launch (environment variable GKS_NVTX=1 at grid creation)
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    struct Rec {
        int group;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    cudaEvent_t open_ev = nullptr;
    // the end event of the last timed launch; the next launch begins at it
    // (one event per launch boundary; whatever the host enqueues between
    // two launches is counted in the second)
    cudaEvent_t last_end = nullptr;
    long launches[K_NGROUPS] = {0};
};

struct gks_grid {
    Ctx c;
    Profiler prof;
    std::string err;
    std::vector<RotorDev> rotors;
    // per rotor: for a share of a neighbouring slab's rotor (gks_share_actuator_lines), the owner
    // grid and the owner's rotor index; else null, -1
    std::vector<std::pair<const gks_grid *, int>> rotor_owner;
    std::vector<BodyDev> bodies;
    std::vector<int> obj_kind, obj_index;
    std::vector<void *> owned;
    double *d_diag = nullptr;
    long nstep = 0;
    bool stepped = false;
    // the FP32 input (FP32C) and max |U|^2 of the current state are in place
    // (left by the last step or state upload): the next step skips its prep
    bool prep_valid = false;
    // gks_step_adjoint: FP32 arithmetic in the local reverse maps
    bool adj_fp32 = false;
    // CUDA graph of one steady-state step (gks_set_graphs): captured when
    // first needed and again after any change of what its launches read by
    // value (inflow, body force, profiling mode), counted by `version`
    bool use_graphs = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;   // capture stream (the grid's own may be the legacy one)
    long version = 0, graph_version = -1;
    long graph_launches[K_NGROUPS] = {0};
};

namespace {

thread_local std::string g_err;

int fail(gks_grid *g, int code, const std::string &msg)
{
    if (g)
        g->err = msg;
    else
        g_err = msg;
    return code;
}

int cuda_check(gks_grid *g, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GKS_OK;
    return fail(g, GKS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct Layout {
    size_t state = 0, work = 0;
    size_t o_wk0 = 0, o_wk1 = 0, o_p = 0, o_fq = 0, o_ff[3] = {0, 0, 0};
    size_t o_ih[3], o_ihf[3], o_h64[3], o_part = 0, o_scal = 0, o_diag = 0;
    long np = 0, nfq = 0, nff[3] = {0, 0, 0};
    int P[3], e1p[3];
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int validate(const gks_grid_desc *d, std::string *msg)
{
    if (!d) { *msg = "null grid description"; return GKS_ERR_ARG; }
    if (d->precision != GKS_FP64 && d->precision != GKS_FP32C) { *msg = "bad precision"; return GKS_ERR_ARG; }
    for (int a = 0; a < 3; ++a) {
        const bool p0 = d->bc[a][0] == GKS_BC_PERIODIC, p1 = d->bc[a][1] == GKS_BC_PERIODIC;
        for (int s = 0; s < 2; ++s)
            if (d->bc[a][s] < GKS_BC_PERIODIC || d->bc[a][s] > GKS_BC_EXCHANGE ||
                (d->bc[a][s] == GKS_BC_EXCHANGE && a != 0)) { *msg = "bad boundary kind"; return GKS_ERR_ARG; }
        if (p0 != p1) { *msg = "periodic must be set on both ends of an axis"; return GKS_ERR_ARG; }
        if (d->n[a] < (p0 ? 1 : 3)) { *msg = "too few cells on an axis"; return GKS_ERR_ARG; }
        if (d->n[a] > (1 << 24)) { *msg = "too many cells on an axis"; return GKS_ERR_ARG; }
        if (!d->faces[a]) { *msg = "null face array"; return GKS_ERR_ARG; }
        for (int i = 0; i < d->n[a]; ++i)
            if (!(d->faces[a][i + 1] > d->faces[a][i])) { *msg = "faces must increase"; return GKS_ERR_ARG; }
    }
    if (!(d->mach > 0.0) || !(d->u_ref > 0.0) || !(d->mu >= 0.0)) { *msg = "bad mach, u_ref or mu"; return GKS_ERR_ARG; }
    if (!(d->dt_fixed > 0.0) && !(d->cfl > 0.0)) { *msg = "need cfl > 0 or dt_fixed > 0"; return GKS_ERR_ARG; }
    if (d->precision == GKS_FP32C && !(d->rho_ref > 0.0)) { *msg = "rho_ref must be > 0"; return GKS_ERR_ARG; }
    // face-tile indices of the flux kernels are 32-bit
    if ((double)(d->n[0] + 1) * (d->n[1] + 1) * (d->n[2] + 1) > 2.0e9) { *msg = "too many cells"; return GKS_ERR_ARG; }
    return GKS_OK;
}

void plan(const gks_grid_desc *d, Layout *L)
{
    const size_t R = d->precision == GKS_FP64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) L->P[a] = d->n[a] + 2 * G;
    const long pn = (long)L->P[0] * L->P[1] * L->P[2];
    L->np = (pn + 63) / 64 * 64;
    L->state = (d->precision == GKS_FP64 ? 4 : 8) * (size_t)L->np * R;
    L->nfq = 0;
    for (int a = 0; a < 3; ++a) {
        const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        // rows of the face box padded to 16 bytes (tensor-map stride rule)
        L->e1p[a] = (d->n[t1] + 4 + 3) / 4 * 4;
        const long nfq = (long)(d->n[a] + 1) * (d->n[t2] + 4) * L->e1p[a];
        if (nfq > L->nfq) L->nfq = nfq;
        // face fluxes are kept for x and y only: the z-face kernel applies
        // the stage update itself (FP64 grids keep the z faces too, for the
        // separate update of their double-single arithmetic)
        L->nff[a] = a == 2 && d->precision != GKS_FP64 ? 0 : (long)(d->n[a] + 1) * d->n[t1] * d->n[t2];
    }
    L->nfq = (L->nfq + 63) / 64 * 64;
    size_t o = 0;
    L->o_wk0 = o;
    if (d->precision == GKS_FP32C) o = align256(o + 4 * (size_t)L->np * 4);
    L->o_wk1 = o; o = align256(o + 4 * (size_t)L->np * R);
    L->o_p = o; o = align256(o + (d->precision == GKS_FP64 ? 4 : 8) * (size_t)L->np * R);
    L->o_fq = o; o = align256(o + 8 * (size_t)L->nfq * R);
    for (int a = 0; a < 3; ++a) { L->o_ff[a] = o; o = align256(o + 8 * (size_t)L->nff[a] * R); }
    for (int a = 0; a < 3; ++a) { L->o_ih[a] = o; o = align256(o + (size_t)L->P[a] * R); }
    for (int a = 0; a < 3; ++a) { L->o_ihf[a] = o; o = align256(o + (size_t)(d->n[a] + 1) * R); }
    for (int a = 0; a < 3; ++a) { L->o_h64[a] = o; o = align256(o + (size_t)L->P[a] * 8); }
    L->o_part = o; o = align256(o + (size_t)kMaxPartials * 8 * 8);
    L->o_scal = o; o = align256(o + sizeof(Scalars));
    L->o_diag = o; o = align256(o + 8 * 8);
    L->work = o;
}

// Padded cell widths of one axis (ghosts wrap or mirror like the state).
std::vector<double> padded_widths(const gks_grid_desc *d, int a)
{
    const int n = d->n[a];
    std::vector<double> h(n + 2 * G);
    for (int i = 0; i < n; ++i) h[i + G] = d->faces[a][i + 1] - d->faces[a][i];
    for (int l = 1; l <= G; ++l) {
        if (d->bc[a][0] == GKS_BC_PERIODIC) {
            h[G - l] = h[G + (((-l) % n) + n) % n];
            h[G + n - 1 + l] = h[G + (n - 1 + l) % n];
        } else {
            h[G - l] = h[G + l - 1];
            h[G + n - 1 + l] = h[G + n - l];
        }
    }
    return h;
}

template <typename R>
int upload(gks_grid *g, void *dst, const std::vector<double> &v)
{
    std::vector<R> t(v.size());
    for (size_t i = 0; i < v.size(); ++i) t[i] = (R)v[i];
    return cuda_check(g, cudaMemcpyAsync(dst, t.data(), t.size() * sizeof(R), cudaMemcpyHostToDevice, g->c.stream),
                      "copy geometry");
}

int check_launch(gks_grid *g, const char *what)
{
    return cuda_check(g, cudaGetLastError(), what);
}

int sync(gks_grid *g) { return cuda_check(g, cudaStreamSynchronize(g->c.stream), "stream synchronize"); }

int read_scalars(gks_grid *g, Scalars *s)
{
    int rc = cuda_check(g, cudaMemcpyAsync(s, g->c.scal, sizeof(Scalars), cudaMemcpyDeviceToHost, g->c.stream),
                        "read scalars");
    if (rc) return rc;
    return sync(g);
}

int device_alloc(gks_grid *g, void **p, size_t bytes)
{
    int rc = cuda_check(g, cudaMalloc(p, bytes), "allocate object buffers");
    if (rc == GKS_OK) g->owned.push_back(*p);
    return rc;
}

cudaEvent_t prof_event(Profiler &p)
{
    if (p.next == p.pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        p.pool.push_back(e);
    }
    return p.pool[p.next++];
}

void prof_mark(void *ctx, int group, int begin)
{
    gks_grid *g = (gks_grid *)ctx;
    Profiler &p = g->prof;
    if (p.nvtx) {
        if (begin)
            nvtxRangePushA(gks_kernel_group_name(group));
        else
            nvtxRangePop();
    }
    if (begin) {
        p.launches[group]++;
        if (p.timing) {
            if (p.last_end) {
                p.open_ev = p.last_end;
            } else {
                p.open_ev = prof_event(p);
                cudaEventRecord(p.open_ev, g->c.stream);
            }
        }
    } else if (p.timing) {
        cudaEvent_t e = prof_event(p);
        cudaEventRecord(e, g->c.stream);
        p.recs.push_back({group, p.open_ev, e});
        p.last_end = e;
    }
}

// Whether the x cells of [lo, hi] (with the one-cell margin of cell_range)
// reach past an exchange side: a kernel support there would need the
// neighbouring slab's cells.
bool reaches_exchange_side(const Ctx &c, double lo, double hi, int side)
{
    if (c.bc[0][side] != GKS_BC_EXCHANGE) return false;
    if (side == 0) return (long)floor((lo - c.x0[0]) / c.hu[0] - 0.5) - 1 - c.xoff < 0;
    return (long)ceil((hi - c.x0[0]) / c.hu[0] - 0.5) + 1 - c.xoff > c.n[0] - 1;
}

bool reaches_exchange(const Ctx &c, double lo, double hi)
{
    return reaches_exchange_side(c, lo, hi, 0) || reaches_exchange_side(c, lo, hi, 1);
}

int cell_range(const Ctx &c, int a, double lo, double hi, int out[2])
{
    const int off = a == 0 ? c.xoff : 0;
    long i0 = (long)floor((lo - c.x0[a]) / c.hu[a] - 0.5) - 1 - off;
    long i1 = (long)ceil((hi - c.x0[a]) / c.hu[a] - 0.5) + 1 - off;
    if (i0 < 0) i0 = 0;
    if (i1 > c.n[a] - 1) i1 = c.n[a] - 1;
    if (i1 < i0) return -1;
    out[0] = (int)i0;
    out[1] = (int)i1;
    return 0;
}

}  // namespace

void gks::record_error(const char *msg) { g_err = msg; }

// Streaming multiprocessors of the current device, looked up once.
int gks::sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

extern "C" {

const char *gks_last_error(const gks_grid *g) { return g ? g->err.c_str() : g_err.c_str(); }

int gks_workspace_bytes(const gks_grid_desc *desc, size_t *state_bytes, size_t *work_bytes)
{
    std::string msg;
    int rc = validate(desc, &msg);
    if (rc) return fail(nullptr, rc, msg);
    if (!state_bytes || !work_bytes) return fail(nullptr, GKS_ERR_ARG, "null output");
    Layout L;
    plan(desc, &L);
    *state_bytes = L.state;
    *work_bytes = L.work;
    return GKS_OK;
}

namespace {

// TMA descriptor of the face box of direction a at `base`: dims (t1 padded,
// t2 + 4, faces, 8 components), box (36, 12, 1, 8). c.e1p must be set.
int encode_face_map(const Ctx &c, int a, void *base, CUtensorMap *out, std::string *msg, int rows = 12)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&encode, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || !encode || q != cudaDriverEntryPointSuccess) {
            encode = nullptr;
            *msg = "cuTensorMapEncodeTiled not available";
            return 1;
        }
    }
    const cuuint64_t es = c.prec == GKS_FP64 ? 8 : 4;
    const int t2 = a == 2 ? 1 : 2;
    const cuuint64_t dims[4] = {(cuuint64_t)c.e1p[a], (cuuint64_t)(c.n[t2] + 4), (cuuint64_t)(c.n[a] + 1), 8};
    const cuuint64_t strides[3] = {dims[0] * es, dims[0] * dims[1] * es, (cuuint64_t)c.nfq * es};
    const cuuint32_t box[4] = {36, (cuuint32_t)rows, 1, 8};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode(out, c.prec == GKS_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *msg = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return 1;
    }
    return 0;
}

}  // namespace

int gks_create_grid(const gks_grid_desc *desc, void *d_state, void *d_work, gks_grid **out)
{
    std::string msg;
    int rc = validate(desc, &msg);
    if (rc) return fail(nullptr, rc, msg);
    if (!out || !d_state || !d_work) return fail(nullptr, GKS_ERR_ARG, "null buffer or output");
    if (((uintptr_t)d_state & 255) || ((uintptr_t)d_work & 255))
        return fail(nullptr, GKS_ERR_ARG, "buffers must be 256-byte aligned");
    Layout L;
    plan(desc, &L);
    gks_grid *g = new gks_grid();
    Ctx &c = g->c;
    c.prec = desc->precision;
    for (int a = 0; a < 3; ++a) {
        c.n[a] = desc->n[a];
        c.P[a] = L.P[a];
        c.bc[a][0] = desc->bc[a][0];
        c.bc[a][1] = desc->bc[a][1];
    }
    c.np = L.np;
    c.ncell = (long)c.n[0] * c.n[1] * c.n[2];
    c.lambda = desc->mach * desc->mach / (2.0 * desc->u_ref * desc->u_ref);
    c.theta = 1.0 / (2.0 * c.lambda);
    c.csound = sqrt(c.theta);
    c.mu = desc->mu;
    c.rho_ref = desc->precision == GKS_FP32C ? desc->rho_ref : 0.0;
    c.off = c.rho_ref;
    c.cfl = desc->cfl;
    c.dt_fixed = desc->dt_fixed;
    c.inflow[0] = 1.0;
    c.inflow[1] = c.inflow[2] = c.inflow[3] = 0.0;
    c.fbody[0] = c.fbody[1] = c.fbody[2] = 0.0;
    c.stream = (cudaStream_t)desc->stream;
    char *w = (char *)d_work;
    c.state = d_state;
    c.wk0 = c.prec == GKS_FP32C ? (void *)(w + L.o_wk0) : d_state;
    c.wk1 = w + L.o_wk1;
    c.pbuf = w + L.o_p;
    c.fq = w + L.o_fq;
    c.nfq = L.nfq;
    for (int a = 0; a < 3; ++a) {
        c.ff[a] = w + L.o_ff[a];
        c.nff[a] = L.nff[a];
        c.ih[a] = w + L.o_ih[a];
        c.ihf[a] = w + L.o_ihf[a];
        c.h64[a] = (double *)(w + L.o_h64[a]);
    }
    c.partials = (double *)(w + L.o_part);
    c.scal = (Scalars *)(w + L.o_scal);
    g->d_diag = (double *)(w + L.o_diag);
    c.staging = (double *)c.ff[0];   // the face-flux buffers hold >= 4 N doubles
    c.mark = prof_mark;
    const char *nv = getenv("GKS_NVTX");
    g->prof.nvtx = nv && nv[0] == '1';
    c.mark_ctx = g;

    // geometry tables
    c.hmin = INFINITY;
    for (int a = 0; a < 3; ++a) {
        std::vector<double> h = padded_widths(desc, a);
        std::vector<double> ih(h.size()), ihf(c.n[a] + 1);
        for (size_t i = 0; i < h.size(); ++i) ih[i] = 1.0 / h[i];
        for (int f = 0; f <= c.n[a]; ++f) ihf[f] = 1.0 / (0.5 * (h[G + f - 1] + h[G + f]));
        for (int i = 0; i < c.n[a]; ++i) c.hmin = fmin(c.hmin, h[G + i]);
        c.x0[a] = desc->faces[a][0];
        c.hu[a] = h[G];
        c.uniform[a] = 1;
        for (int i = 0; i < c.n[a]; ++i)
            if (fabs(h[G + i] - h[G]) > 1e-12 * fabs(h[G])) c.uniform[a] = 0;
        if (c.prec == GKS_FP64) {
            rc = upload<double>(g, c.ih[a], ih);
            if (!rc) rc = upload<double>(g, c.ihf[a], ihf);
        } else {
            rc = upload<float>(g, c.ih[a], ih);
            if (!rc) rc = upload<float>(g, c.ihf[a], ihf);
        }
        if (!rc) rc = upload<double>(g, c.h64[a], h);
        if (rc) { msg = g->err; delete g; return fail(nullptr, rc, msg); }
    }
    // TMA descriptors of the face box, one per direction
    for (int a = 0; a < 3; ++a) {
        c.e1p[a] = L.e1p[a];
        std::string m;
        if (encode_face_map(c, a, c.fq, &c.tmap[a], &m) ||
            (c.prec == GKS_FP32C && encode_face_map(c, a, c.fq, &c.tmapT[a], &m, 20))) {
            delete g;
            return fail(nullptr, GKS_ERR_CUDA, m);
        }
    }
    rc = cuda_check(g, cudaMemsetAsync(c.scal, 0, sizeof(Scalars), c.stream), "clear scalars");
    if (!rc) rc = cuda_check(g, cudaMemsetAsync(c.state, 0, L.state, c.stream), "clear state");
    if (!rc) rc = cuda_check(g, cudaMemsetAsync(w, 0, L.o_ff[0], c.stream), "clear work");
    if (!rc) {
        launch_fill_rest(c);
        rc = check_launch(g, "fill state");
    }
    if (!rc) rc = sync(g);
    if (rc) { msg = g->err; delete g; return fail(nullptr, rc, msg); }
    *out = g;
    return GKS_OK;
}

int gks_destroy_grid(gks_grid *g)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    cudaStreamSynchronize(g->c.stream);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (void *p : g->owned) cudaFree(p);
    for (cudaEvent_t e : g->prof.pool) cudaEventDestroy(e);
    delete g;
    return GKS_OK;
}

int gks_set_stream(gks_grid *g, void *stream)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    g->c.stream = (cudaStream_t)stream;
    return GKS_OK;
}

int gks_set_state(gks_grid *g, const double *h_state)
{
    if (!g || !h_state) return fail(g, GKS_ERR_ARG, "null argument");
    int rc = cuda_check(g, cudaMemcpyAsync(g->c.staging, h_state, sizeof(double) * 4 * g->c.ncell,
                                           cudaMemcpyHostToDevice, g->c.stream),
                        "copy state to device");
    if (rc) return rc;
    launch_scatter_state_prep(g->c, g->c.staging);
    g->prep_valid = true;
    return check_launch(g, "scatter state");
}

int gks_get_state(gks_grid *g, double *h_state)
{
    if (!g || !h_state) return fail(g, GKS_ERR_ARG, "null argument");
    launch_gather_state(g->c, g->c.staging);
    int rc = check_launch(g, "gather state");
    if (!rc)
        rc = cuda_check(g, cudaMemcpyAsync(h_state, g->c.staging, sizeof(double) * 4 * g->c.ncell,
                                           cudaMemcpyDeviceToHost, g->c.stream),
                        "copy state to host");
    if (!rc) rc = sync(g);
    return rc;
}

int gks_set_inflow(gks_grid *g, double rho, double u, double v, double w)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    if (!(rho > 0.0)) return fail(g, GKS_ERR_ARG, "inflow density must be > 0");
    g->c.inflow[0] = rho;
    g->c.inflow[1] = u;
    g->c.inflow[2] = v;
    g->c.inflow[3] = w;
    g->version++;
    return GKS_OK;
}

int gks_set_body_force(gks_grid *g, double fx, double fy, double fz)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    g->c.fbody[0] = fx;
    g->c.fbody[1] = fy;
    g->c.fbody[2] = fz;
    g->version++;
    return GKS_OK;
}

int gks_add_actuator_lines(gks_grid *g, const gks_rotor_desc *d, int *id)
{
    if (!g || !d || !id) return fail(g, GKS_ERR_ARG, "null argument");
    Ctx &c = g->c;
    if (g->stepped) return fail(g, GKS_ERR_STATE, "objects must be added before the first step");
    if (!(c.uniform[0] && c.uniform[1] && c.uniform[2])) return fail(g, GKS_ERR_ARG, "actuator lines need uniform axes");
    if (d->n_blades < 1 || d->n_blades > GKS_MAX_BLADES || d->n_pts < 1 || !(d->eps > 0.0) || !d->r ||
        !d->chord || !d->twist || !d->width || !(d->radius > 0.0) || !(d->u_inf_ref > 0.0) || !(d->rho_inf > 0.0))
        return fail(g, GKS_ERR_ARG, "bad rotor description");
    const int nb = d->n_blades, np = d->n_pts, npts = nb * np;
    RotorDev r;
    memset(&r, 0, sizeof(r));
    r.nb = nb;
    r.np = np;
    r.correction = d->correction ? 1 : 0;
    r.tip = d->tip_correction ? 1 : 0;
    {
        // g1 = exp(-c1 (N lambda - c2)) + 0.1 of the tip factors, lambda = omega R / U_inf
        const double c1[2] = {0.1219, 0.0984}, c2[2] = {21.52, 13.026};
        const double tsr = d->omega * d->radius / d->u_inf_ref;
        for (int k = 0; k < 2; ++k) r.tip_g[k] = exp(-c1[k] * (d->n_blades * tsr - c2[k])) + 0.1;
    }
    for (int a = 0; a < 3; ++a) r.hub[a] = d->hub[a];
    r.omega = d->omega;
    r.az0 = d->azimuth0;
    r.radius = d->radius;
    r.eps = d->eps;
    r.rho_inf = d->rho_inf;
    r.uref = d->u_inf_ref;
    double rmax = 0.0, rmin = INFINITY;
    for (int p = 0; p < np; ++p) {
        rmax = fmax(rmax, d->r[p]);
        rmin = fmin(rmin, d->r[p]);
    }
    r.rmin = rmin;
    r.rmax = rmax;
    rmax = fmax(fabs(rmax), fabs(rmin));
    const double cut = 3.0 * d->eps;
    if (cell_range(c, 0, d->hub[0] - cut, d->hub[0] + cut, r.box[0]) ||
        cell_range(c, 1, d->hub[1] - rmax - cut, d->hub[1] + rmax + cut, r.box[1]) ||
        cell_range(c, 2, d->hub[2] - rmax - cut, d->hub[2] + rmax + cut, r.box[2]))
        return fail(g, GKS_ERR_RANGE, "rotor outside the grid");
    r.norm = 1.0 / (d->eps * d->eps * d->eps * pow(3.14159265358979323846, 1.5));
    r.ie2 = 1.0 / (d->eps * d->eps);
    // per point: scale, X (3), F (4), Xr (3 floats in 2 doubles)
    const size_t nd = 4 * (size_t)np + (size_t)npts + 3 * (size_t)npts + 4 * (size_t)npts + 2 * (size_t)npts +
                      2 * nb + 2 * nb + 3;
    double *buf = nullptr;
    int rc = device_alloc(g, (void **)&buf, nd * sizeof(double));
    if (rc) return rc;
    std::vector<double> host(nd, 0.0);
    size_t o = 0;
    r.r = buf + o; memcpy(&host[o], d->r, np * sizeof(double)); o += np;
    r.chord = buf + o; memcpy(&host[o], d->chord, np * sizeof(double)); o += np;
    r.twist = buf + o; memcpy(&host[o], d->twist, np * sizeof(double)); o += np;
    r.width = buf + o; memcpy(&host[o], d->width, np * sizeof(double)); o += np;
    r.scale = buf + o; for (int q = 0; q < npts; ++q) host[o + q] = 1.0; o += npts;
    r.X = buf + o; o += 3 * (size_t)npts;
    r.F = buf + o; o += 4 * (size_t)npts;
    r.Xr = reinterpret_cast<float *>(buf + o); o += 2 * (size_t)npts;
    r.et = buf + o; o += 2 * nb;
    r.out = buf + o;
    rc = cuda_check(g, cudaMemcpyAsync(buf, host.data(), nd * sizeof(double), cudaMemcpyHostToDevice, c.stream),
                    "copy rotor");
    if (!rc) rc = sync(g);
    if (rc) return rc;
    g->rotors.push_back(r);
    g->rotor_owner.push_back({nullptr, -1});
    g->obj_kind.push_back(0);
    g->obj_index.push_back((int)g->rotors.size() - 1);
    *id = (int)g->obj_kind.size() - 1;
    return GKS_OK;
}

int gks_set_slab_lattice(gks_grid *g, double x0, double hx, int cells_before)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    Ctx &c = g->c;
    if (g->stepped || !g->obj_kind.empty())
        return fail(g, GKS_ERR_STATE, "the slab lattice is set before rotors, bodies and steps");
    if (!(hx > 0.0) || cells_before < 0 || !c.uniform[0]) return fail(g, GKS_ERR_ARG, "bad slab lattice");
    // the slab's first face lies on that lattice
    if (fabs(c.x0[0] - (x0 + cells_before * hx)) > 1e-6 * hx || fabs(c.hu[0] - hx) > 1e-6 * hx)
        return fail(g, GKS_ERR_ARG, "the slab's x faces are not on that lattice");
    c.x0[0] = x0;
    c.hu[0] = hx;
    c.xoff = cells_before;
    return GKS_OK;
}

int gks_share_actuator_lines(gks_grid *owner, int id, gks_grid *g, int *id_out)
{
    if (!owner || !g || !id_out || owner == g) return fail(g, GKS_ERR_ARG, "bad arguments");
    if (id < 0 || id >= (int)owner->obj_kind.size() || owner->obj_kind[id] != 0)
        return fail(g, GKS_ERR_ARG, "no rotor with that id on the owner");
    const int ri = owner->obj_index[id];
    if (owner->rotor_owner[ri].first) return fail(g, GKS_ERR_ARG, "that rotor is itself a share");
    Ctx &c = g->c;
    if (g->stepped) return fail(g, GKS_ERR_STATE, "objects must be added before the first step");
    if (c.prec != owner->c.prec || !(c.uniform[0] && c.uniform[1] && c.uniform[2]) ||
        c.x0[0] != owner->c.x0[0] || c.hu[0] != owner->c.hu[0])
        return fail(g, GKS_ERR_ARG, "the sharing slab needs the owner's precision and x lattice");
    RotorDev r = owner->rotors[ri];   // the owner's point buffers, read after the owner's loads
    r.shared = 1;
    const double cut = 3.0 * r.eps, rm = fmax(fabs(r.rmax), fabs(r.rmin));
    if (cell_range(c, 0, r.hub[0] - cut, r.hub[0] + cut, r.box[0]) ||
        cell_range(c, 1, r.hub[1] - rm - cut, r.hub[1] + rm + cut, r.box[1]) ||
        cell_range(c, 2, r.hub[2] - rm - cut, r.hub[2] + rm + cut, r.box[2]))
        return fail(g, GKS_ERR_RANGE, "the rotor's support misses this slab");
    g->rotors.push_back(r);
    g->rotor_owner.push_back({owner, ri});
    g->obj_kind.push_back(0);
    g->obj_index.push_back((int)g->rotors.size() - 1);
    *id_out = (int)g->obj_kind.size() - 1;
    return GKS_OK;
}

int gks_set_force_scales(gks_grid *g, int id, const double *h_scales)
{
    if (!g || !h_scales || id < 0 || id >= (int)g->obj_kind.size() || g->obj_kind[id] != 0)
        return fail(g, GKS_ERR_ARG, "bad rotor id or scales");
    const RotorDev &r = g->rotors[g->obj_index[id]];
    return cuda_check(g, cudaMemcpyAsync(r.scale, h_scales, sizeof(double) * r.nb * r.np, cudaMemcpyHostToDevice,
                                         g->c.stream),
                      "copy force scales");
}

int gks_add_ib_points(gks_grid *g, int n, const double *xyz, const double *dS, const double *vel, double eps,
                      int niter, double tol, int *id)
{
    if (!g || !xyz || !dS || !id) return fail(g, GKS_ERR_ARG, "null argument");
    Ctx &c = g->c;
    if (g->stepped) return fail(g, GKS_ERR_STATE, "objects must be added before the first step");
    if (!(c.uniform[0] && c.uniform[1] && c.uniform[2])) return fail(g, GKS_ERR_ARG, "immersed bodies need uniform axes");
    if (n < 1 || !(eps > 0.0) || niter < 1 || niter > 1000 || !(tol >= 0.0)) return fail(g, GKS_ERR_ARG, "bad body description");
    BodyDev b;
    memset(&b, 0, sizeof(b));
    b.n = n;
    b.niter = niter;
    b.eps = eps;
    b.tol = tol;
    if (body_box(c, xyz, n, eps, b.box)) return fail(g, GKS_ERR_RANGE, "body outside the grid");
    {
        double lo = INFINITY, hi = -INFINITY;
        for (int p = 0; p < n; ++p) {
            lo = fmin(lo, xyz[3 * p]);
            hi = fmax(hi, xyz[3 * p]);
        }
        if (reaches_exchange(c, lo - 3.0 * eps, hi + 3.0 * eps))
            return fail(g, GKS_ERR_RANGE, "body support reaches an exchange side of the slab");
    }
    b.nbox = (long)(b.box[0][1] - b.box[0][0] + 1) * (b.box[1][1] - b.box[1][0] + 1) * (b.box[2][1] - b.box[2][0] + 1);
    const size_t nd = 7 * (size_t)n + 8 * (size_t)b.nbox + 7 + niter;
    double *buf = nullptr;
    int rc = device_alloc(g, (void **)&buf, nd * sizeof(double));
    if (rc) return rc;
    std::vector<double> host(7 * (size_t)n, 0.0);
    memcpy(&host[0], xyz, 3 * n * sizeof(double));
    if (vel) memcpy(&host[3 * (size_t)n], vel, 3 * n * sizeof(double));
    memcpy(&host[6 * (size_t)n], dS, n * sizeof(double));
    b.xyz = buf;
    b.vel = buf + 3 * (size_t)n;
    b.dS = buf + 6 * (size_t)n;
    b.Vbar = buf + 7 * (size_t)n;
    b.vbar = b.Vbar + b.nbox;
    b.phi = b.vbar + 3 * b.nbox;
    b.fsum = b.phi + b.nbox;
    b.out = b.fsum + 3 * b.nbox;
    rc = cuda_check(g, cudaMemcpyAsync(buf, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream),
                    "copy body");
    if (!rc) rc = cuda_check(g, cudaMemsetAsync(b.Vbar, 0, (8 * (size_t)b.nbox + 7 + niter) * sizeof(double), c.stream),
                             "clear body");
    if (rc) return rc;
    launch_body_precompute(c, b);
    rc = check_launch(g, "body fields");
    if (rc) return rc;
    // CSR of the back-interpolation weights: count, scan on the host, fill
    long *d_cnt = nullptr;
    rc = device_alloc(g, (void **)&d_cnt, sizeof(long) * (n + 1));
    if (rc) return rc;
    launch_body_csr_count(c, b, d_cnt);
    std::vector<long> cnt(n), off(n + 1, 0);
    rc = check_launch(g, "count weights");
    if (!rc) rc = cuda_check(g, cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(long) * n, cudaMemcpyDeviceToHost, c.stream),
                             "read counts");
    if (!rc) rc = sync(g);
    if (rc) return rc;
    for (int p = 0; p < n; ++p) off[p + 1] = off[p] + cnt[p];
    b.nnz = off[n];
    b.csr_off = d_cnt;
    char *cbuf = nullptr;
    rc = device_alloc(g, (void **)&cbuf, (size_t)b.nnz * (sizeof(double) + sizeof(int) + sizeof(float)) +
                                             3 * (sizeof(double) + sizeof(float)) * b.nbox + 64);
    if (rc) return rc;
    b.csr_w = (double *)cbuf;
    b.Ubox = b.csr_w + b.nnz;
    b.csr_cell = (int *)(b.Ubox + 3 * b.nbox);
    b.csr_wf = (float *)(b.csr_cell + b.nnz);
    b.Uboxf = b.csr_wf + b.nnz;
    rc = cuda_check(g, cudaMemcpyAsync(d_cnt, off.data(), sizeof(long) * (n + 1), cudaMemcpyHostToDevice, c.stream),
                    "copy offsets");
    if (rc) return rc;
    launch_body_csr_fill(c, b);
    rc = check_launch(g, "fill weights");
    if (!rc) rc = sync(g);
    if (rc) return rc;
    g->bodies.push_back(b);
    g->obj_kind.push_back(1);
    g->obj_index.push_back((int)g->bodies.size() - 1);
    *id = (int)g->obj_kind.size() - 1;
    return GKS_OK;
}

namespace {
int check_flags(gks_grid *g, int flags, const char *where);

// Per stage st of a recorded step, the Gauss-point inputs of every
// direction go to the tape.
void use_tape_gauss(Ctx &cc, const AdjWork &w, int st)
{
    cc.ngp = w.nG;
    cc.gp_bytes = w.gp_bytes;
    for (int d = 0; d < 3; ++d) cc.gp_dir[d] = w.gps[st][d];
}

// One S2O4 step of the grid with its forcing. With a tape (FP64 grids) the
// step also keeps what its reverse reads: t_n and dt, the ghost-filled W^n
// and W*, the state before the forcing, and both stages' Gauss-point
// inputs; the arithmetic of the step is the same either way.
int step_once(gks_grid *g, const AdjWork *tp)
{
    Ctx &c = g->c;
    Ctx cc = c;
    const int nobj = (int)g->obj_kind.size();
    const bool fused_prep = nobj <= 8;
    const size_t bytes4 = sizeof(double) * 4 * c.np;
    int rc = GKS_OK;
    g->prof.last_end = nullptr;   // launch boundaries are shared inside a step only
    if (!g->prep_valid) launch_prep(c);
    launch_ghost(c, c.wk0);
    launch_cfl(c);   // dt from max |U|^2, which it clears
    if (tp) {
        rc = cuda_check(g, cudaMemcpyAsync(tp->hdr + 1, &c.scal->t, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                           c.stream), "record time");
        if (!rc) rc = cuda_check(g, cudaMemsetAsync(tp->hdr, kTapeMagicByte, sizeof(double), c.stream), "mark tape");
        const double gb = tp->gp_bytes;
        if (!rc) rc = cuda_check(g, cudaMemcpyAsync(tp->hdr + 3, &gb, sizeof(double), cudaMemcpyHostToDevice, c.stream),
                                 "record the tape's storage");
        if (rc) return rc;
        if (c.prec == GKS_FP64) {
            rc = cuda_check(g, cudaMemcpyAsync(tp->A0, c.wk0, bytes4, cudaMemcpyDeviceToDevice, c.stream), "record W^n");
            if (rc) return rc;
            cc.wk1 = tp->Ws;
        } else {
            // FP32C: the FP32 input (rho - off) as the reverse's stencil reads
            // it, and as FP64 with rho for the rest of the reverse
            rc = cuda_check(g, cudaMemcpyAsync(tp->A0f, c.wk0, sizeof(float) * 4 * c.np, cudaMemcpyDeviceToDevice,
                                               c.stream), "record the FP32 W^n");
            if (rc) return rc;
            launch_widen(c, (const float *)c.wk0, nullptr, tp->A0, 4 * c.np, c.np, c.off);
        }
        if (c.prec == GKS_FP64) use_tape_gauss(cc, *tp, 0);
    }
    launch_stage(cc, 1);
    launch_ghost(cc, cc.wk1);
    if (tp) {
        if (c.prec == GKS_FP32C) {
            rc = cuda_check(g, cudaMemcpyAsync(tp->Wsf, c.wk1, sizeof(float) * 4 * c.np, cudaMemcpyDeviceToDevice,
                                               c.stream), "record the FP32 W*");
            if (rc) return rc;
            launch_widen(c, (const float *)c.wk1, nullptr, tp->Ws, 4 * c.np, c.np, c.off);
        } else {
            use_tape_gauss(cc, *tp, 1);
        }
    }
    // stage 2 also prepares the next step on every cell outside the forcing
    // boxes; the boxes are prepared again after the forcing
    if (fused_prep) {
        cc.prep_next = 1;
        cc.nprep_box = nobj;
        for (int k = 0; k < nobj; ++k) {
            const int(*box)[2] = g->obj_kind[k] == 0 ? g->rotors[g->obj_index[k]].box : g->bodies[g->obj_index[k]].box;
            memcpy(cc.prep_box[k], box, sizeof(int) * 6);
        }
    }
    launch_stage(cc, 2);
    if (tp && c.prec == GKS_FP64 &&
        (rc = cuda_check(g, cudaMemcpyAsync(tp->Wp, c.state, bytes4, cudaMemcpyDeviceToDevice, c.stream),
                         "record the state before the forcing")))
        return rc;
    if (tp && c.prec == GKS_FP32C)
        launch_widen(c, (const float *)c.state, (const float *)c.state + 4 * c.np, tp->Wp, 4 * c.np, 0, 0.0);
    for (size_t k = 0; k < g->obj_kind.size(); ++k)
        if (g->obj_kind[k] == 0) launch_alm(c, g->rotors[g->obj_index[k]]);
    for (size_t k = 0; k < g->obj_kind.size(); ++k)
        if (g->obj_kind[k] == 1) {
            const int bi = g->obj_index[k];
            launch_ibm(c, g->bodies[bi]);
            if (tp && (rc = cuda_check(g, cudaMemcpyAsync(tp->hdr + 4 + bi, g->bodies[bi].out + 3, sizeof(double),
                                                          cudaMemcpyDeviceToDevice, c.stream),
                                       "record the IBM iterations")))
                return rc;
        }
    if (fused_prep)
        for (int k = 0; k < nobj; ++k) launch_prep_box(c, cc.prep_box[k]);
    g->prep_valid = fused_prep;
    launch_advance(c);
    g->prof.last_end = nullptr;
    rc = check_launch(g, "step");
    if (rc) return rc;
    g->nstep++;
    return GKS_OK;
}

// Debug-bounds builds: whether a kernel met an index outside its buffer
// since the last look (always false in a plain build).
bool bounds_hit()
{
    const int f = bounds_flag_stencil() | bounds_flag_forcing() | bounds_flag_adjoint();
    return f != 0;
}

int finish_steps(gks_grid *g, double *t_out)
{
    Scalars sc;
    int rc = read_scalars(g, &sc);
    if (rc) return rc;
    if (bounds_hit()) return fail(g, GKS_ERR_DEBUG_BOUNDS, "a kernel met an index outside its buffer");
    if (t_out) *t_out = sc.t;
    if (sc.flags) {
        int flags = 0;
        cudaMemcpyAsync(&g->c.scal->flags, &flags, sizeof(int), cudaMemcpyHostToDevice, g->c.stream);
        sync(g);
        return check_flags(g, sc.flags, "state");
    }
    return GKS_OK;
}

int check_flags(gks_grid *g, int flags, const char *where)
{
    std::string w(where);
    if (flags & FLAG_NONFINITE) return fail(g, GKS_ERR_NONFINITE, "non-finite value in the " + w);
    if (flags & FLAG_RANGE) return fail(g, GKS_ERR_RANGE, "actuator point outside the sampled interior");
    if (flags & FLAG_CFL) return fail(g, GKS_ERR_CFL, "fixed time step above the CFL limit");
    if (flags & FLAG_TIMEOUT) return fail(g, GKS_ERR_CUDA, "a device-side wait timed out");
    return flags ? fail(g, GKS_ERR_CUDA, "device flag raised in the " + w) : GKS_OK;
}
}  // namespace

namespace {
// Capture one step (as step_once enqueues it in the current host state) into
// the grid's graph. Nothing runs; the host-side effects of the captured step
// (step count, launch counters) are undone, a replay redoes them.
int capture_step(gks_grid *g)
{
    Ctx &c = g->c;
    int rc = GKS_OK;
    if (!g->cap_stream &&
        (rc = cuda_check(g, cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking), "capture stream")))
        return rc;
    long saved[K_NGROUPS];
    memcpy(saved, g->prof.launches, sizeof(saved));
    const long nstep0 = g->nstep;
    const cudaStream_t own = c.stream;
    c.stream = g->cap_stream;
    rc = cuda_check(g, cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) {
        c.stream = own;
        return rc;
    }
    rc = step_once(g, nullptr);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c.stream, &graph);
    c.stream = own;
    g->nstep = nstep0;
    for (int k = 0; k < K_NGROUPS; ++k) {
        g->graph_launches[k] = g->prof.launches[k] - saved[k];
        g->prof.launches[k] = saved[k];
    }
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc ? rc : cuda_check(g, e, "end capture");
    }
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->gexec = nullptr;
    g->graph = graph;
    rc = cuda_check(g, cudaGraphInstantiate(&g->gexec, graph, 0), "instantiate graph");
    if (rc) return rc;
    g->graph_version = g->version;
    return GKS_OK;
}
}  // namespace

int gks_set_fp64_arithmetic(gks_grid *g, int double_single)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    if (g->c.prec != GKS_FP64) return fail(g, GKS_ERR_STATE, "FP64 grids only");
    g->c.fp64_ds = double_single != 0;
    g->version++;   // a captured step graph is captured again
    return GKS_OK;
}

int gks_set_graphs(gks_grid *g, int on)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    g->use_graphs = on != 0;
    return GKS_OK;
}

int gks_step_async(gks_grid *g, int nsteps)
{
    if (!g || nsteps < 0) return fail(g, GKS_ERR_ARG, "bad arguments");
    for (const auto &o : g->rotor_owner)
        if (o.first) return fail(g, GKS_ERR_STATE, "a slab holding a share of another slab's rotor steps with its group");
    for (int s = 0; s < nsteps; ++s) {
        // a step replays the graph in the steady state: the next step's
        // prep done by the last step (at most kMaxPrepBoxes forcing
        // objects), no per-launch profiling, and one plain step done before
        // (the kernels' one-time launch setup)
        const bool replay = g->use_graphs && g->stepped && g->prep_valid && g->obj_kind.size() <= 8 &&
                            !g->prof.timing && !g->prof.nvtx;
        int rc;
        if (replay) {
            if (!g->gexec || g->graph_version != g->version) {
                rc = capture_step(g);
                if (rc) return rc;
            }
            rc = cuda_check(g, cudaGraphLaunch(g->gexec, g->c.stream), "graph launch");
            if (rc) return rc;
            for (int k = 0; k < K_NGROUPS; ++k) g->prof.launches[k] += g->graph_launches[k];
            g->nstep++;
        } else {
            g->stepped = true;
            rc = step_once(g, nullptr);
            if (rc) return rc;
        }
    }
    return GKS_OK;
}

int gks_sync(gks_grid *g, double *t_out)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    return finish_steps(g, t_out);
}

int gks_step(gks_grid *g, int nsteps, double *t_out)
{
    int rc = gks_step_async(g, nsteps);
    return rc ? rc : finish_steps(g, t_out);
}

namespace {
// Slab groups: the x halo exchange of the working array of a stage (0: W,
// 1: W*) between every pair of neighbouring slabs, in both directions.
void slab_exchange(gks_grid *const *sl, int n, int stage)
{
    auto work = [&](int s) { return stage == 0 ? sl[s]->c.wk0 : sl[s]->c.wk1; };
    for (int s = 0; s < n; ++s) {
        if (sl[s]->c.bc[0][1] != GKS_BC_EXCHANGE) continue;
        const int r = s + 1 < n ? s + 1 : 0;   // the right neighbour; slab 0 closes a periodic x axis
        launch_halo_copy(sl[s]->c, work(s), 1, sl[r]->c, work(r), 0);
        launch_halo_copy(sl[r]->c, work(r), 0, sl[s]->c, work(s), 1);
    }
}

// One step of a slab group on one stream: the sequence of step_once on every
// slab, with the halo exchange after each ghost fill and the group's largest
// |U|^2 for the time step.
int slab_step_once(gks_grid *const *sl, int n)
{
    for (int s = 0; s < n; ++s) {
        gks_grid *g = sl[s];
        g->prof.last_end = nullptr;
        g->stepped = true;
        if (!g->prep_valid) launch_prep(g->c);
        launch_ghost(g->c, g->c.wk0);
    }
    slab_exchange(sl, n, 0);
    Scalars *scal[64];
    for (int s = 0; s < n; ++s) scal[s] = sl[s]->c.scal;
    launch_group_max_u2(scal, n, sl[0]->c.stream);
    for (int s = 0; s < n; ++s) launch_cfl(sl[s]->c);
    std::vector<Ctx> cc(n);
    for (int s = 0; s < n; ++s) {
        cc[s] = sl[s]->c;
        launch_stage(cc[s], 1);
        launch_ghost(cc[s], cc[s].wk1);
    }
    slab_exchange(sl, n, 1);
    std::vector<int> fused(n);
    for (int s = 0; s < n; ++s) {
        gks_grid *g = sl[s];
        const int nobj = (int)g->obj_kind.size();
        fused[s] = nobj <= 8;
        if (fused[s]) {
            cc[s].prep_next = 1;
            cc[s].nprep_box = nobj;
            for (int k = 0; k < nobj; ++k) {
                const int(*box)[2] =
                    g->obj_kind[k] == 0 ? g->rotors[g->obj_index[k]].box : g->bodies[g->obj_index[k]].box;
                memcpy(cc[s].prep_box[k], box, sizeof(int) * 6);
            }
        }
        launch_stage(cc[s], 2);
    }
    // rotors: each owner's loads and projection, then every share's projection
    // of the owner's point forces into its own cells; then the bodies
    for (int s = 0; s < n; ++s)
        for (size_t k = 0; k < sl[s]->obj_kind.size(); ++k)
            if (sl[s]->obj_kind[k] == 0 && !sl[s]->rotors[sl[s]->obj_index[k]].shared)
                launch_alm(sl[s]->c, sl[s]->rotors[sl[s]->obj_index[k]]);
    for (int s = 0; s < n; ++s)
        for (size_t k = 0; k < sl[s]->obj_kind.size(); ++k)
            if (sl[s]->obj_kind[k] == 0 && sl[s]->rotors[sl[s]->obj_index[k]].shared)
                launch_alm_spread(sl[s]->c, sl[s]->rotors[sl[s]->obj_index[k]]);
    for (int s = 0; s < n; ++s) {
        gks_grid *g = sl[s];
        const Ctx &c = g->c;
        for (size_t k = 0; k < g->obj_kind.size(); ++k)
            if (g->obj_kind[k] == 1) launch_ibm(c, g->bodies[g->obj_index[k]]);
        if (fused[s])
            for (int k = 0; k < cc[s].nprep_box; ++k) launch_prep_box(c, cc[s].prep_box[k]);
        g->prep_valid = fused[s];
        launch_advance(c);
        g->prof.last_end = nullptr;
        const int rc = check_launch(g, "slab step");
        if (rc) return rc;
        g->nstep++;
    }
    return GKS_OK;
}

// Host copy of a device array of doubles (slab-group checks).
int fetch(gks_grid *g, const double *d, size_t n, std::vector<double> *out)
{
    out->resize(n);
    return cuda_check(g, cudaMemcpy(out->data(), d, n * sizeof(double), cudaMemcpyDeviceToHost), "read widths");
}

// The x geometry tables of two neighbouring slabs at their cut: the ghost
// cell widths of each exchange side become the other slab's interior widths
// (at creation they mirror the slab's own), and the inverse widths of those
// ghosts and the inverse centre distance of the cut face follow, as a grid of
// the whole domain has them.
int patch_cut(gks_grid *gl, gks_grid *gr)
{
    Ctx &l = gl->c, &r = gr->c;
    std::vector<double> hl, hr0;
    int rc = fetch(gl, l.h64[0], l.P[0], &hl);
    if (!rc && gr != gl) rc = fetch(gr, r.h64[0], r.P[0], &hr0);
    if (rc) return rc;
    std::vector<double> &hr = gr == gl ? hl : hr0;   // one slab closing a periodic axis on itself
    const int nl = l.n[0];
    for (int k = 0; k < G; ++k) {
        hl[G + nl + k] = hr[G + k];
        hr[G - 1 - k] = hl[G + nl - 1 - k];
    }
    std::vector<double> il(hl.size()), ir(hr.size()), fl(nl + 1), fr(r.n[0] + 1);
    for (size_t i = 0; i < hl.size(); ++i) il[i] = 1.0 / hl[i];
    for (size_t i = 0; i < hr.size(); ++i) ir[i] = 1.0 / hr[i];
    for (int f = 0; f <= nl; ++f) fl[f] = 1.0 / (0.5 * (hl[G + f - 1] + hl[G + f]));
    for (int f = 0; f <= r.n[0]; ++f) fr[f] = 1.0 / (0.5 * (hr[G + f - 1] + hr[G + f]));
    const bool f64 = l.prec == GKS_FP64;
    rc = upload<double>(gl, l.h64[0], hl);
    if (!rc) rc = upload<double>(gr, r.h64[0], hr);
    if (!rc) rc = f64 ? upload<double>(gl, l.ih[0], il) : upload<float>(gl, l.ih[0], il);
    if (!rc) rc = f64 ? upload<double>(gr, r.ih[0], ir) : upload<float>(gr, r.ih[0], ir);
    if (!rc) rc = f64 ? upload<double>(gl, l.ihf[0], fl) : upload<float>(gl, l.ihf[0], fl);
    if (!rc) rc = f64 ? upload<double>(gr, r.ihf[0], fr) : upload<float>(gr, r.ihf[0], fr);
    if (!rc) rc = sync(gl);
    return rc;
}
}  // namespace

int gks_slab_step(gks_grid *const *slabs, int nslab, int nsteps, double *t_out)
{
    if (!slabs || nslab < 1 || nslab > 64 || nsteps < 0) return fail(nullptr, GKS_ERR_ARG, "bad slab-group arguments");
    for (int s = 0; s < nslab; ++s)
        if (!slabs[s]) return fail(nullptr, GKS_ERR_ARG, "null slab");
    gks_grid *g0 = slabs[0];
    const Ctx &c0 = g0->c;
    std::vector<double> hy0, hz0;
    int rc = fetch(g0, c0.h64[1], c0.P[1], &hy0);
    if (!rc) rc = fetch(g0, c0.h64[2], c0.P[2], &hz0);
    if (rc) return rc;
    double hmin = INFINITY;
    for (int s = 0; s < nslab; ++s) {
        gks_grid *g = slabs[s];
        const Ctx &c = g->c;
        if (c.prec != c0.prec || c.fp64_ds != c0.fp64_ds || c.n[1] != c0.n[1] || c.n[2] != c0.n[2] ||
            c.stream != c0.stream || c.lambda != c0.lambda || c.mu != c0.mu || c.off != c0.off || c.cfl != c0.cfl ||
            c.dt_fixed != c0.dt_fixed)
            return fail(nullptr, GKS_ERR_ARG, "slabs differ in precision, arithmetic, y/z cells, physics or stream");
        for (int a = 1; a < 3; ++a)
            if (c.bc[a][0] != c0.bc[a][0] || c.bc[a][1] != c0.bc[a][1])
                return fail(nullptr, GKS_ERR_ARG, "slabs differ in their y or z boundary kinds");
        if (g->use_graphs) return fail(nullptr, GKS_ERR_ARG, "slab groups step without CUDA graphs");
        std::vector<double> hy, hz;
        rc = fetch(g, c.h64[1], c.P[1], &hy);
        if (!rc) rc = fetch(g, c.h64[2], c.P[2], &hz);
        if (rc) return rc;
        if (hy != hy0 || hz != hz0) return fail(nullptr, GKS_ERR_ARG, "slabs differ in their y or z faces");
        const bool hi_ex = c.bc[0][1] == GKS_BC_EXCHANGE;
        const bool lo_next = slabs[s + 1 < nslab ? s + 1 : 0]->c.bc[0][0] == GKS_BC_EXCHANGE;
        if (s + 1 < nslab && !(hi_ex && lo_next))
            return fail(nullptr, GKS_ERR_ARG, "neighbouring slabs must face each other with exchange sides");
        if (s + 1 == nslab && hi_ex != lo_next)
            return fail(nullptr, GKS_ERR_ARG, "a periodic x axis needs exchange sides on both ends of the group");
        if (hi_ex) {
            gks_grid *gr = slabs[s + 1 < nslab ? s + 1 : 0];
            rc = patch_cut(g, gr);
            if (rc) return rc;
        }
        hmin = fmin(hmin, c.hmin);
    }
    // forcing: the slabs place cells on one x lattice, and a rotor whose
    // support reaches an exchange side is shared with the slab behind it
    const bool forced = [&] {
        for (int s = 0; s < nslab; ++s)
            if (!slabs[s]->obj_kind.empty()) return true;
        return false;
    }();
    if (forced) {
        int before = 0;
        for (int s = 0; s < nslab; ++s) {
            const Ctx &c = slabs[s]->c;
            if (c.x0[0] != c0.x0[0] || c.hu[0] != c0.hu[0] || c.xoff != before)
                return fail(nullptr, GKS_ERR_ARG, "forcing in a slab group needs every slab on one x lattice "
                                                  "(gks_set_slab_lattice)");
            before += c.n[0];
        }
        for (int s = 0; s < nslab; ++s) {
            gks_grid *g = slabs[s];
            for (size_t k = 0; k < g->rotors.size(); ++k) {
                const RotorDev &r = g->rotors[k];
                if (r.shared) continue;
                const double cut = 3.0 * r.eps;
                for (int side = 0; side < 2; ++side) {
                    if (!reaches_exchange_side(g->c, r.hub[0] - cut, r.hub[0] + cut, side)) continue;
                    const gks_grid *nb = slabs[side == 0 ? (s > 0 ? s - 1 : nslab - 1) : (s + 1 < nslab ? s + 1 : 0)];
                    bool covered = false;
                    for (const auto &o : nb->rotor_owner) covered |= o.first == g && o.second == (int)k;
                    if (!covered)
                        return fail(nullptr, GKS_ERR_RANGE, "a rotor support reaches a slab cut and the slab behind "
                                                            "it holds no share of it (gks_share_actuator_lines)");
                }
            }
        }
    }
    for (int s = 0; s < nslab; ++s) slabs[s]->c.hmin = hmin;   // the CFL step of the whole domain
    for (int k = 0; k < nsteps; ++k) {
        rc = slab_step_once(slabs, nslab);
        if (rc) return rc;
    }
    for (int s = 0; s < nslab; ++s) {
        rc = finish_steps(slabs[s], s == 0 ? t_out : nullptr);
        if (rc) {
            g_err = slabs[s]->err;
            return rc;
        }
    }
    return GKS_OK;
}

int gks_get_time(gks_grid *g, double *t, double *dt_last)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    Scalars sc;
    int rc = read_scalars(g, &sc);
    if (rc) return rc;
    if (t) *t = sc.t;
    if (dt_last) *dt_last = sc.dt;
    return GKS_OK;
}

int gks_set_time(gks_grid *g, double t)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    int rc = cuda_check(g, cudaMemcpyAsync(&g->c.scal->t, &t, sizeof(double), cudaMemcpyHostToDevice, g->c.stream),
                        "set time");
    if (!rc) rc = sync(g);
    return rc;
}

int gks_forces(gks_grid *g, int id, gks_forces_out *out, double *h_points)
{
    if (!g || !out || id < 0 || id >= (int)g->obj_kind.size()) return fail(g, GKS_ERR_ARG, "bad object id");
    memset(out, 0, sizeof(*out));
    int rc = sync(g);
    if (rc) return rc;
    if (g->obj_kind[id] == 0) {
        const RotorDev &r = g->rotors[g->obj_index[id]];
        std::vector<double> o(2 * r.nb + 3);
        rc = cuda_check(g, cudaMemcpy(o.data(), r.out, o.size() * sizeof(double), cudaMemcpyDeviceToHost), "read loads");
        if (rc) return rc;
        out->kind = 0;
        out->n_blades = r.nb;
        for (int b = 0; b < r.nb; ++b) {
            out->thrust[b] = o[b];
            out->torque[b] = o[r.nb + b];
        }
        out->power = o[2 * r.nb];
        out->cp = o[2 * r.nb + 1];
        out->ct = o[2 * r.nb + 2];
        if (h_points)
            rc = cuda_check(g, cudaMemcpy(h_points, r.F, 4 * sizeof(double) * r.nb * r.np, cudaMemcpyDeviceToHost),
                            "read point loads");
        return rc;
    }
    const BodyDev &b = g->bodies[g->obj_index[id]];
    std::vector<double> o(7 + b.niter);
    rc = cuda_check(g, cudaMemcpy(o.data(), b.out, o.size() * sizeof(double), cudaMemcpyDeviceToHost), "read body force");
    if (rc) return rc;
    out->kind = 1;
    for (int d = 0; d < 3; ++d) out->body_force[d] = o[d];
    out->iters = (int)o[3];
    out->residual = o[4];
    if (h_points) memcpy(h_points, &o[7], sizeof(double) * b.niter);
    return GKS_OK;
}

int gks_forces_record_len(const gks_grid *g, int id, size_t *n)
{
    if (!g || !n || id < 0 || id >= (int)g->obj_kind.size()) return fail(nullptr, GKS_ERR_ARG, "bad object id");
    if (g->obj_kind[id] == 0)
        *n = 2 * (size_t)g->rotors[g->obj_index[id]].nb + 3;
    else
        *n = 7 + (size_t)g->bodies[g->obj_index[id]].niter;
    return GKS_OK;
}

int gks_forces_async(gks_grid *g, int id, double *h_out, size_t n)
{
    size_t len = 0;
    if (!g || !h_out) return fail(g, GKS_ERR_ARG, "null argument");
    int rc = gks_forces_record_len(g, id, &len);
    if (rc) return fail(g, rc, "bad object id");
    if (n < len) return fail(g, GKS_ERR_ARG, "record buffer too small");
    const double *src = g->obj_kind[id] == 0 ? g->rotors[g->obj_index[id]].out : g->bodies[g->obj_index[id]].out;
    return cuda_check(g, cudaMemcpyAsync(h_out, src, sizeof(double) * len, cudaMemcpyDeviceToHost, g->c.stream),
                      "copy load record");
}

int gks_diagnostics(gks_grid *g, double out[5])
{
    if (!g || !out) return fail(g, GKS_ERR_ARG, "null argument");
    // timed as its own range of the misc group (no boundary shared with a step)
    g->prof.last_end = nullptr;
    mark(g->c, K_MISC, 1);
    launch_diagnostics(g->c, g->d_diag);
    mark(g->c, K_MISC, 0);
    g->prof.last_end = nullptr;
    int rc = check_launch(g, "diagnostics");
    if (!rc)
        rc = cuda_check(g, cudaMemcpyAsync(out, g->d_diag, 5 * sizeof(double), cudaMemcpyDeviceToHost, g->c.stream),
                        "read diagnostics");
    if (!rc) rc = sync(g);
    return rc;
}

namespace {
struct BlobHeader {
    char magic[8];
    int prec, n[3];
    double t;
    long nstep;
    size_t payload;
};
size_t payload_bytes(const Ctx &c) { return (size_t)c.ncell * (c.prec == GKS_FP64 ? 4 * 8 : 8 * 4); }
}  // namespace

int gks_checkpoint_bytes(gks_grid *g, size_t *bytes)
{
    if (!g || !bytes) return fail(g, GKS_ERR_ARG, "null argument");
    *bytes = sizeof(BlobHeader) + payload_bytes(g->c);
    return GKS_OK;
}

int gks_save_state(gks_grid *g, void *h_blob, size_t bytes)
{
    if (!g || !h_blob) return fail(g, GKS_ERR_ARG, "null argument");
    const size_t pb = payload_bytes(g->c);
    if (bytes < sizeof(BlobHeader) + pb) return fail(g, GKS_ERR_ARG, "blob too small");
    Scalars sc;
    int rc = read_scalars(g, &sc);
    if (rc) return rc;
    BlobHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "GKSCKPT1", 8);
    h.prec = g->c.prec;
    for (int a = 0; a < 3; ++a) h.n[a] = g->c.n[a];
    h.t = sc.t;
    h.nstep = g->nstep;
    h.payload = pb;
    memcpy(h_blob, &h, sizeof(h));
    launch_raw_copy(g->c, g->c.staging, 1);
    rc = check_launch(g, "gather checkpoint");
    if (!rc)
        rc = cuda_check(g, cudaMemcpyAsync((char *)h_blob + sizeof(h), g->c.staging, pb, cudaMemcpyDeviceToHost, g->c.stream),
                        "copy checkpoint");
    if (!rc) rc = sync(g);
    return rc;
}

int gks_load_state(gks_grid *g, const void *h_blob, size_t bytes)
{
    if (!g || !h_blob || bytes < sizeof(BlobHeader)) return fail(g, GKS_ERR_ARG, "bad blob");
    BlobHeader h;
    memcpy(&h, h_blob, sizeof(h));
    if (memcmp(h.magic, "GKSCKPT1", 8) != 0 || h.prec != g->c.prec || h.n[0] != g->c.n[0] || h.n[1] != g->c.n[1] ||
        h.n[2] != g->c.n[2] || h.payload != payload_bytes(g->c) || bytes < sizeof(h) + h.payload)
        return fail(g, GKS_ERR_ARG, "checkpoint does not match this grid");
    int rc = cuda_check(g, cudaMemcpyAsync(g->c.staging, (const char *)h_blob + sizeof(h), h.payload,
                                           cudaMemcpyHostToDevice, g->c.stream),
                        "copy checkpoint");
    if (rc) return rc;
    launch_raw_copy(g->c, g->c.staging, 0);
    g->prep_valid = false;
    rc = check_launch(g, "scatter checkpoint");
    if (rc) return rc;
    rc = cuda_check(g, cudaMemcpyAsync(&g->c.scal->t, &h.t, sizeof(double), cudaMemcpyHostToDevice, g->c.stream),
                    "set time");
    if (!rc) rc = sync(g);
    g->nstep = h.nstep;
    return rc;
}

int gks_set_state_device(gks_grid *g, const double *d_state)
{
    if (!g || !d_state) return fail(g, GKS_ERR_ARG, "null argument");
    launch_scatter_state_prep(g->c, d_state);
    g->prep_valid = true;
    return check_launch(g, "scatter state");
}

int gks_get_state_device(gks_grid *g, double *d_state)
{
    if (!g || !d_state) return fail(g, GKS_ERR_ARG, "null argument");
    launch_gather_state(g->c, d_state);
    return check_launch(g, "gather state");
}

namespace {
long total_points(const gks_grid *g)
{
    long n = 0;
    for (const RotorDev &r : g->rotors) n += (long)r.nb * r.np;
    return n;
}

// Storage of the tape's Gauss-point inputs: the compute type of the reverse
// (FP32 for the FP32 forward of FP32C grids).
int gp_bytes_of(const gks_grid *g) { return (g->adj_fp32 || g->c.prec == GKS_FP32C) ? 4 : 8; }

// tape_path: recorded steps, which also cover FP32C grids.
int adjoint_check(gks_grid *g, bool tape_path)
{
    const Ctx &c = g->c;
    if (c.prec != GKS_FP64 && c.prec != GKS_FP32C) return fail(g, GKS_ERR_STATE, "bad grid precision for the adjoint");
    if (!(c.dt_fixed > 0.0)) return fail(g, GKS_ERR_STATE, "the adjoint needs a fixed time step (dt_fixed > 0)");
    for (const BodyDev &b : g->bodies)
        if (b.tol > 0.0 && !tape_path)
            return fail(g, GKS_ERR_STATE,
                        "gks_step_adjoint covers immersed bodies with a fixed iteration count (tol = 0); "
                        "recorded steps cover the tolerance mode");
    if (tape_path && g->bodies.size() > (size_t)kTapeMaxBodies)
        return fail(g, GKS_ERR_STATE, "too many immersed bodies for a tape");
    if (g->rotors.size() > 1) return fail(g, GKS_ERR_STATE, "the adjoint covers at most one rotor");
    if (c.bc[0][0] == GKS_BC_EXCHANGE || c.bc[0][1] == GKS_BC_EXCHANGE)
        return fail(g, GKS_ERR_STATE, "the adjoint covers whole grids, not slabs");
    // the reverse t2 gather indexes its 64 face arrays with 32-bit offsets
    for (int d = 0; d < 3; ++d) {
        const double nf = (double)(c.n[d] + 1) * c.n[(d + 1) % 3] * c.n[(d + 2) % 3];
        if (64.0 * nf >= 2147483647.0) return fail(g, GKS_ERR_ARG, "grid too large for the adjoint");
    }
    return GKS_OK;
}
}  // namespace

int gks_set_adjoint_precision(gks_grid *g, int precision)
{
    if (!g || (precision != GKS_FP64 && precision != GKS_FP32C)) return fail(g, GKS_ERR_ARG, "bad adjoint precision");
    g->adj_fp32 = precision == GKS_FP32C;
    return GKS_OK;
}

int gks_adjoint_workspace_bytes(const gks_grid *g, size_t *bytes)
{
    if (!g || !bytes) return fail(nullptr, GKS_ERR_ARG, "null argument");
    *bytes = adjoint_bytes(g->c, total_points(g), gp_bytes_of(g));
    return GKS_OK;
}

int gks_adjoint_tape_bytes(const gks_grid *g, size_t *bytes)
{
    if (!g || !bytes) return fail(nullptr, GKS_ERR_ARG, "null argument");
    AdjWork w;
    *bytes = adjoint_tape_carve(g->c, gp_bytes_of(g), nullptr, &w);
    return GKS_OK;
}

int gks_adjoint_scratch_bytes(const gks_grid *g, size_t *bytes)
{
    if (!g || !bytes) return fail(nullptr, GKS_ERR_ARG, "null argument");
    AdjWork w;
    *bytes = adjoint_scratch_carve(g->c, total_points(g), nullptr, &w);
    return GKS_OK;
}

namespace {
// The reverse of one step from the tape in w (recorded by gks_step_record
// or by the recompute of gks_step_adjoint), with the time of the tape.
// init_sc: set the private scalars from the tape (the recompute of
// gks_step_adjoint has set them already, and its flags are kept).
int reverse_from_tape(gks_grid *g, const AdjWork &w, bool init_sc, double t_n, double dt, const int *ibm_iters,
                      const double *d_adj_np1, double *d_adj_n, double power_seed, double *h_grad_scales,
                      double *h_grad_uinf)
{
    const Ctx &c = g->c;
    Ctx cc = c;
    cc.mark = nullptr;
    cc.scal = w.sc;
    cc.wk1 = w.Ws;
    if (c.prec == GKS_FP32C) {
        // the tape holds FP64 arrays with rho (not rho - off): the reverse
        // runs as on an FP64 grid, with the FP32 inverse widths of the forward
        cc.prec = GKS_FP64;
        cc.off = 0.0;
        for (int d = 0; d < 3; ++d) {
            launch_widen(cc, (const float *)c.ih[d], nullptr, w.ih64[d], c.P[d], 0, 0.0);
            launch_widen(cc, (const float *)c.ihf[d], nullptr, w.ihf64[d], c.n[d] + 1, 0, 0.0);
            cc.ih[d] = w.ih64[d];
            cc.ihf[d] = w.ihf64[d];
        }
    }
    int rc = GKS_OK;
    if (init_sc) {
        rc = cuda_check(g, cudaMemsetAsync(w.sc, 0, sizeof(Scalars), c.stream), "clear reverse scalars");
        if (!rc) rc = cuda_check(g, cudaMemcpyAsync(&w.sc->t, w.hdr + 1, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                                    c.stream), "reverse time");
    }
    if (!rc) rc = cuda_check(g, cudaMemsetAsync(w.scal, 0, 8 * sizeof(double), c.stream), "clear adjoint scalars");
    if (rc) return rc;
    // the rotor loads at t_{n+1} from the state before the forcing
    const RotorDev *rot = g->rotors.empty() ? nullptr : &g->rotors[0];
    if (rot) {
        cc.state = w.Wp;
        launch_alm_loads(cc, *rot);
    }
    cc.state = w.lamP;
    launch_scatter_state(cc, d_adj_np1);
    adjoint_reverse(cc, w, rot, g->bodies.data(), (int)g->bodies.size(), ibm_iters, power_seed, dt, t_n + dt);
    cc.state = w.lamW;
    launch_gather_state(cc, d_adj_n);
    rc = check_launch(g, "adjoint step");
    if (rc) return rc;
    const long npts = total_points(g);
    std::vector<double> pts(8 * (npts > 0 ? npts : 1));
    double gu = 0.0;
    int flags = 0;
    if (npts > 0)
        rc = cuda_check(g, cudaMemcpyAsync(pts.data(), w.pts, sizeof(double) * 8 * npts, cudaMemcpyDeviceToHost, c.stream),
                        "read scale gradients");
    if (!rc) rc = cuda_check(g, cudaMemcpyAsync(&gu, w.scal, sizeof(double), cudaMemcpyDeviceToHost, c.stream),
                             "read inflow gradient");
    if (!rc) rc = cuda_check(g, cudaMemcpyAsync(&flags, &w.sc->flags, sizeof(int), cudaMemcpyDeviceToHost, c.stream),
                             "read reverse flags");
    if (!rc) rc = sync(g);
    if (rc) return rc;
    if (bounds_hit()) return fail(g, GKS_ERR_DEBUG_BOUNDS, "a kernel met an index outside its buffer");
    if (flags) return check_flags(g, flags, "adjoint step");
    if (h_grad_scales)
        for (long q = 0; q < npts; ++q) h_grad_scales[q] += pts[8 * q + 2];
    if (h_grad_uinf) *h_grad_uinf += gu;
    return GKS_OK;
}
}  // namespace

int gks_step_record(gks_grid *g, void *d_tape, double *t_out)
{
    if (!g || !d_tape) return fail(g, GKS_ERR_ARG, "null argument");
    if ((uintptr_t)d_tape & 255) return fail(g, GKS_ERR_ARG, "tape must be 256-byte aligned");
    int rc = adjoint_check(g, true);
    if (rc) return rc;
    AdjWork w;
    adjoint_tape_carve(g->c, gp_bytes_of(g), d_tape, &w);
    g->stepped = true;
    rc = step_once(g, &w);
    if (rc) return rc;
    return finish_steps(g, t_out);
}

int gks_step_reverse(gks_grid *g, void *d_tape, void *d_scratch, const double *d_adj_np1, double *d_adj_n,
                     double power_seed, double *h_grad_scales, double *h_grad_uinf)
{
    if (!g || !d_tape || !d_scratch || !d_adj_np1 || !d_adj_n) return fail(g, GKS_ERR_ARG, "null argument");
    if (((uintptr_t)d_tape | (uintptr_t)d_scratch) & 255)
        return fail(g, GKS_ERR_ARG, "tape and scratch must be 256-byte aligned");
    int rc = adjoint_check(g, true);
    if (rc) return rc;
    AdjWork w;
    adjoint_tape_carve(g->c, gp_bytes_of(g), d_tape, &w);
    adjoint_scratch_carve(g->c, total_points(g), d_scratch, &w);
    double hdr[kTapeHeader];
    rc = cuda_check(g, cudaMemcpyAsync(hdr, w.hdr, sizeof(hdr), cudaMemcpyDeviceToHost, g->c.stream), "read tape");
    if (!rc) rc = sync(g);
    if (rc) return rc;
    unsigned char magic[sizeof(double)];
    memcpy(magic, hdr, sizeof(magic));
    for (unsigned char m : magic)
        if (m != kTapeMagicByte) return fail(g, GKS_ERR_STATE, "tape not recorded");
    if (hdr[3] != (double)w.gp_bytes)
        return fail(g, GKS_ERR_STATE, "tape recorded with another adjoint precision");
    w.c32 = &g->c;
    std::vector<int> iters(g->bodies.size());
    for (size_t k = 0; k < iters.size(); ++k) {
        iters[k] = (int)hdr[4 + k];
        if (iters[k] < 1 || iters[k] > g->bodies[k].niter)
            return fail(g, GKS_ERR_STATE, "tape with an invalid IBM iteration count");
    }
    return reverse_from_tape(g, w, true, hdr[1], hdr[2], iters.data(), d_adj_np1, d_adj_n, power_seed,
                             h_grad_scales, h_grad_uinf);
}

int gks_step_adjoint(gks_grid *g, void *d_adj_work, double t_n, const double *d_state_n, const double *d_adj_np1,
                     double *d_adj_n, double power_seed, double *h_grad_scales, double *h_grad_uinf)
{
    if (!g || !d_adj_work || !d_state_n || !d_adj_np1 || !d_adj_n) return fail(g, GKS_ERR_ARG, "null argument");
    if ((uintptr_t)d_adj_work & 255) return fail(g, GKS_ERR_ARG, "adjoint workspace must be 256-byte aligned");
    int rc = adjoint_check(g, false);
    if (rc) return rc;
    const Ctx &c = g->c;
    AdjWork w;
    adjoint_carve(c, total_points(g), gp_bytes_of(g), d_adj_work, &w);
    const double dt = c.dt_fixed;
    // forward recompute of the step from W^n into the tape part of the
    // workspace, on private scalars (the grid's time and state stay as they
    // are): A0 = G(W^n), W* = G(stage 1), Wp = stage 2 before the forcing
    Ctx cc = c;
    cc.mark = nullptr;
    cc.scal = w.sc;
    const double hv[3] = {t_n, dt, (double)w.gp_bytes};
    rc = cuda_check(g, cudaMemsetAsync(w.sc, 0, sizeof(Scalars), c.stream), "clear reverse scalars");
    if (!rc) rc = cuda_check(g, cudaMemcpyAsync(&w.sc->t, hv, 2 * sizeof(double), cudaMemcpyHostToDevice, c.stream),
                             "set time");
    if (!rc) rc = cuda_check(g, cudaMemcpyAsync(w.hdr + 1, hv, sizeof(hv), cudaMemcpyHostToDevice, c.stream),
                             "record time");
    if (!rc) rc = cuda_check(g, cudaMemsetAsync(w.hdr, kTapeMagicByte, sizeof(double), c.stream), "mark tape");
    if (rc) return rc;
    if (c.prec == GKS_FP32C) {
        // the FP32C step recomputed in the workspace: the compensated state
        // (hi, lo) in the scratch's lamA (cleared by the reverse before its
        // use), P in the tape's Ws as hi, lo floats until W* is widened into
        // it after stage 2, the FP32 reconstruction inputs of both stages in
        // A0f and Wsf as the reverse reads them
        w.c32 = &g->c;
        cc.state = w.lamA;
        cc.wk0 = w.A0f;
        cc.wk1 = w.Wsf;
        cc.pbuf = w.Ws;
        cc.prep_next = 0;
        launch_scatter_state_prep(cc, d_state_n);
        launch_ghost(cc, cc.wk0);
        launch_widen(cc, w.A0f, nullptr, w.A0, 4 * c.np, c.np, c.off);
        launch_stage(cc, 1);
        launch_ghost(cc, cc.wk1);
        launch_stage(cc, 2);
        launch_widen(cc, w.Wsf, nullptr, w.Ws, 4 * c.np, c.np, c.off);
        launch_widen(cc, (const float *)w.lamA, (const float *)w.lamA + 4 * c.np, w.Wp, 4 * c.np, 0, 0.0);
    } else {
        cc.state = w.A0;
        cc.wk0 = w.A0;
        cc.wk1 = w.Ws;
        launch_scatter_state(cc, d_state_n);
        launch_ghost(cc, w.A0);
        use_tape_gauss(cc, w, 0);
        launch_stage(cc, 1);
        launch_ghost(cc, cc.wk1);
        cc.state = w.Wp;
        use_tape_gauss(cc, w, 1);
        launch_stage(cc, 2);
    }
    std::vector<int> iters(g->bodies.size());
    for (size_t k = 0; k < iters.size(); ++k) iters[k] = g->bodies[k].niter;   // tol = 0: every iteration runs
    return reverse_from_tape(g, w, false, t_n, dt, iters.data(), d_adj_np1, d_adj_n, power_seed, h_grad_scales,
                             h_grad_uinf);
}

int gks_profile_enable(gks_grid *g, int timing_on)
{
    if (!g) return fail(nullptr, GKS_ERR_ARG, "null grid");
    int rc = sync(g);
    if (rc) return rc;
    Profiler &p = g->prof;
    p.timing = timing_on != 0;
    g->version++;
    p.next = 0;
    p.last_end = nullptr;
    p.recs.clear();
    for (int k = 0; k < K_NGROUPS; ++k) p.launches[k] = 0;
    return GKS_OK;
}

int gks_profile_read(gks_grid *g, gks_profile_out *out)
{
    if (!g || !out) return fail(g, GKS_ERR_ARG, "null argument");
    int rc = sync(g);
    if (rc) return rc;
    Profiler &p = g->prof;
    memset(out, 0, sizeof(*out));
    for (const Profiler::Rec &r : p.recs) {
        float ms = 0.0f;
        rc = cuda_check(g, cudaEventElapsedTime(&ms, r.a, r.b), "event time");
        if (rc) return rc;
        out->ms[r.group] += ms;
    }
    for (int k = 0; k < K_NGROUPS; ++k) {
        out->launches[k] = p.launches[k];
        out->total_launches += p.launches[k];
        p.launches[k] = 0;
    }
    p.next = 0;
    p.last_end = nullptr;
    p.recs.clear();
    return GKS_OK;
}

const char *gks_kernel_group_name(int group)
{
    static const char *names[K_NGROUPS] = {"prep", "ghost", "cfl", "face_eq", "face_flux",
                                           "flux_update", "alm", "ibm", "misc"};
    return (group >= 0 && group < K_NGROUPS) ? names[group] : "";
}

int gks_state_layout(const gks_grid *g, long out[7])
{
    if (!g || !out) return fail(nullptr, GKS_ERR_ARG, "null argument");
    out[0] = g->c.P[0];
    out[1] = g->c.P[1];
    out[2] = g->c.P[2];
    out[3] = g->c.prec == GKS_FP64 ? 8 : 4;
    out[4] = g->c.prec == GKS_FP64 ? 4 : 8;
    out[5] = g->c.np;
    out[6] = G;
    return GKS_OK;
}

}  // extern "C"
