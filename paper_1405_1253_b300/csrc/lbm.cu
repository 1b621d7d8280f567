// lbm.cu -- C ABI of the B300 D2Q37 thermal lattice Boltzmann library (include/lbm.h).
//
// One translation unit: the kernels live in the included .cuh files; this file holds the
// context, argument validation, launch configuration and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "common.cuh"
#include "step_f64.cuh"
#include "step_ff.cuh"
#include "step_f32.cuh"
#include "step_f32dev.cuh"
#include "init_diag.cuh"
#include "adjoint.cuh"
#include "adjoint_ff.cuh"
#include "walls.cuh"
#include "adjoint_walls.cuh"
#include "ensemble.cuh"
#include "selftest.cuh"
#include "probe.cuh"

using namespace lbm;

// ---------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(LBM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

#define LAUNCH_CHECK() CU(cudaGetLastError())

// Selects a device for the scope and restores the caller's current device on exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && (prev == dev || cudaSetDevice(dev) == cudaSuccess)) ok = true;
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------------
// Device allocations of the library go through dev_malloc / dev_malloc_async, so that a test
// can refuse the n-th next one (lbm_test_fail_alloc) and check that every caller reports
// LBM_ENOMEM and leaves nothing half-built.
// ---------------------------------------------------------------------------------
static std::atomic<int> g_fail_alloc{-1};

static bool alloc_refused() {
    int n = g_fail_alloc.load();
    while (n >= 0)
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 0;
    return false;
}

template <class T>
static cudaError_t dev_malloc(T** p, size_t bytes) {
    if (alloc_refused()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void**)p, bytes);
}

template <class T>
static cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t st) {
    if (alloc_refused()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync((void**)p, bytes, st);
}

// ---------------------------------------------------------------------------------
// Lattice constants: solved once on the host, uploaded once per device.
// ---------------------------------------------------------------------------------
static std::mutex g_lat_mutex;
static bool g_quad_done = false;
static Quadrature g_quad;
static bool g_dev_uploaded[128];

// Shell weights for kernel parameters; valid once a context exists (the quadrature is
// solved before the first context is created and never changes afterwards).
static const double* quad_w_shell() { return g_quad.w_shell; }

static int host_quadrature(Quadrature* out) {
    std::lock_guard<std::mutex> lk(g_lat_mutex);
    if (!g_quad_done) {
        g_quad = solve_quadrature_host();
        g_quad_done = true;
    }
    if (!g_quad.ok) return fail(LBM_ECUDA, "quadrature solve did not converge");
    *out = g_quad;
    return LBM_OK;
}

static void split3(long double v, float (&t)[3]) {
    t[0] = (float)v;
    t[1] = (float)(v - (long double)t[0]);
    t[2] = (float)(v - (long double)t[0] - (long double)t[1]);
}

static int upload_lattice(int dev) {
    Quadrature q;
    int rc = host_quadrature(&q);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_lat_mutex);
    if (dev < 0 || dev >= 128) return fail(LBM_EINVAL, "device index %d out of range", dev);
    if (g_dev_uploaded[dev]) return LBM_OK;
    DevLattice h{};
    for (int s = 0; s < NSHELL; s++) {
        h.w[s] = q.w_shell[s];
        h.wf[s] = (float)q.w_shell[s];
    }
    h.r = q.r;
    h.r2 = q.r * q.r;
    h.r2_half = 0.5 * h.r2;
    h.r_hi = (float)h.r;
    h.r2_hi = (float)h.r2;
    const long double rl = q.r, r2l = rl * rl;
    split3(rl, h.r3);
    split3(6.0L * r2l, h.r2x6);
    split3(12.0L * r2l, h.r2x12);
    split3(3.0L * r2l * r2l, h.r4x3);
    CU(cudaMemcpyToSymbol(d_lat, &h, sizeof h));
    PairInfo pairs[NPAIR];
    for (int k = 0; k < NPAIR; k++) {
        const int A = pair_first(k);
        pairs[k] = PairInfo{A, opp(A), cx(A), cz(A), (float)cx(A), (float)cz(A), (float)c2(A)};
    }
    CU(cudaMemcpyToSymbol(d_pairs, pairs, sizeof pairs));
    int sfirst[NSHELL] = {0}, snp[NSHELL] = {0}, vel[Q][2];
    for (int k = NPAIR - 1; k >= 0; k--) { sfirst[shell_of(pair_first(k))] = k; snp[shell_of(pair_first(k))]++; }
    for (int l = 0; l < Q; l++) { vel[l][0] = cx(l); vel[l][1] = cz(l); }
    CU(cudaMemcpyToSymbol(d_shell_first, sfirst, sizeof sfirst));
    CU(cudaMemcpyToSymbol(d_shell_npair, snp, sizeof snp));
    {   // shell groups (common.cuh): |c|^2 = (1, 2), (4, 8), (5, 10), then 9 across both lanes
        const int gs[NGROUP][2] = {{1, 2}, {3, 5}, {4, 7}, {6, 6}};
        ShellGroup g[NGROUP];
        for (int i = 0; i < NGROUP; i++) {
            const int a = gs[i][0], b = gs[i][1];
            if (a != b) {
                if (snp[a] != snp[b]) return fail(LBM_ECUDA, "shell group %d: unequal pair counts", i);
                g[i] = ShellGroup{sfirst[a], sfirst[b], snp[a], a, b, (float)shell_c2(a), (float)shell_c2(b)};
            } else {
                if (snp[a] != 2) return fail(LBM_ECUDA, "shell group %d: the lone shell needs two pairs", i);
                g[i] = ShellGroup{sfirst[a], sfirst[a] + 1, 1, a, a, (float)shell_c2(a), (float)shell_c2(a)};
            }
        }
        CU(cudaMemcpyToSymbol(d_groups, g, sizeof g));
    }
    CU(cudaMemcpyToSymbol(d_vel, vel, sizeof vel));
    CU(cudaDeviceSynchronize());
    g_dev_uploaded[dev] = true;
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------------
struct lbm_ctx {
    int Lx, Lz, prec;
    double tau, grav;
    void* buf[2];
    size_t bytes;
    int cur;                    // index of the buffer holding the current state
    cudaStream_t stream;
    int device;
    // private scratch
    double* zcol = nullptr;     // 2 * Lx interface heights / per-column adjoint sums
    double* modes = nullptr;    // 4 * modes_cap mode parameters
    int modes_cap = 0;
    double* part = nullptr;     // reduction partials
    size_t part_cap = 0;        // in doubles
    double* small = nullptr;    // Lz + 8 doubles (Tbar, widths, sums)
    double* dLrow = nullptr;    // Lz doubles (width gradient)
    double* colred = nullptr;   // 2 * Lx (init adjoint per-column sums)
    unsigned int* err = nullptr;  // device error word
    // host-buffer stepping (lbm_step_host): copy streams and their events, made on first use
    // (NCOPY streams per direction, each copying one part of the state)
    cudaStream_t s_in[2] = {nullptr, nullptr}, s_out[2] = {nullptr, nullptr};
    cudaEvent_t e_in[2] = {nullptr, nullptr}, e_out[2] = {nullptr, nullptr}, e_step = nullptr;
    // wall rule: 0 half-way bounce-back, 1 thermal walls (lbm_set_walls)
    int thermal = 0;
    ThermalWall tw{};
    double* gmu = nullptr;      // 6 * Q * Lx: ghost-pull scratch of the thermal-wall adjoint
    // LBM_F32_DEV: the per-row reference (step_f32dev.cuh)
    double* fref = nullptr;     // Q * Lz: fref_l(z) (FP64)
    float* dref = nullptr;      // NDREF * Lz: gref_l(z) - fref_l(z) by (shell, c_z) class
    float* rowc = nullptr;      // RC_N * Lz: per-row constants (RC_N per row)
};

static size_t pop_bytes(int prec) { return (prec == LBM_F64 || prec == LBM_F64_FF) ? 8 : 4; }
static bool valid_prec(int prec) {
    return prec == LBM_F64 || prec == LBM_F32 || prec == LBM_F32_DEV || prec == LBM_F64_FF;
}

static StepParams step_params(const lbm_ctx* c) {
    StepParams p;
    p.Lx = c->Lx;
    p.Lz = c->Lz;
    p.plane = c->Lx * c->Lz;
    p.omega = 1.0 / c->tau;
    p.one_m_omega = 1.0 - 1.0 / c->tau;
    p.us_z = -(c->grav * c->tau);
    p.T_shift = ((c->grav * c->grav) * c->tau) * (1.0 - c->tau) / DIM;   // exactly 0 for g = 0
    p.grav = c->grav;
    return p;
}

static int ensure_part(lbm_ctx* c, size_t n) {
    if (c->part_cap >= n) return LBM_OK;
    if (c->part) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->part);
    }
    c->part = nullptr;
    c->part_cap = 0;
    if (dev_malloc(&c->part, n * sizeof(double)) != cudaSuccess)
        return fail(LBM_ENOMEM, "cannot allocate %zu reduction doubles", n);
    c->part_cap = n;
    return LBM_OK;
}

static void free_ctx(lbm_ctx* c) {
    if (!c) return;
    void* ps[] = {c->zcol, c->modes, c->part, c->small, c->dLrow, c->colred, c->err, c->gmu,
                  c->fref, c->dref, c->rowc};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (int k = 0; k < 2; k++) {
        for (cudaStream_t st : {c->s_in[k], c->s_out[k]})
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t ev : {c->e_in[k], c->e_out[k]})
            if (ev) cudaEventDestroy(ev);
    }
    if (c->e_step) cudaEventDestroy(c->e_step);
    delete c;
}

// One step of the columns of tiling t in precision prec (p describes the buffers); not for
// LBM_F32_DEV, whose step needs its context's reference (ctx_step).
static void launch_step(int prec, const void* fin, void* fout, const StepParams& p, const Tiling& t,
                        cudaStream_t st) {
    switch (prec) {
        case LBM_F64: launch_step_f64((const double*)fin, (double*)fout, p, t, st); break;
        case LBM_F64_FF: launch_step_ff((const double*)fin, (double*)fout, p, quad_w_shell(), t, st); break;
        default: launch_step_f32((const float*)fin, (float*)fout, p, t, st); break;
    }
}

// One step of context c from fin to fout with its wall rule (one launch either way).
static void ctx_step(const lbm_ctx* c, const void* fin, void* fout, const StepParams& p, cudaStream_t st) {
    const Tiling t = make_tiling(p.Lx, p.Lz, BLOCK_Z);
    if (c->prec == LBM_F32_DEV) {        // bounce-back walls only (lbm_set_walls)
        launch_step_f32dev((const float*)fin, (float*)fout, fd_params(p, c->dref, c->rowc), t, st);
        return;
    }
    if (!c->thermal) {
        launch_step(c->prec, fin, fout, p, t, st);
        return;
    }
    const int blocks = tiling_blocks(t);
    switch (c->prec) {
        case LBM_F64:
            k_step_f64_thermal<<<blocks, BLOCK_Z, 0, st>>>((const double*)fin, (double*)fout, p, t, c->tw);
            break;
        case LBM_F64_FF:
            launch_pdl(k_step_ff_thermal, blocks, BLOCK_Z, st, (const double*)fin, (double*)fout,
                       ff_params(p, quad_w_shell()), t, c->tw);
            break;
        default:
            k_step_f32_thermal<<<blocks, BLOCK_Z, 0, st>>>((const float*)fin, (float*)fout, f32_params(p), t, c->tw);
            break;
    }
}

#define NOT_DEV(c, what)                                                                        \
    do {                                                                                        \
        if ((c)->prec == LBM_F32_DEV) return fail(LBM_ESTATE, what " is not available for LBM_F32_DEV"); \
    } while (0)

#define NEED_BOUNCE_BACK(c, what)                                                               \
    do {                                                                                        \
        if ((c)->thermal) return fail(LBM_ESTATE, what " supports the bounce-back walls only"); \
    } while (0)

template <class S>
static void launch_moments(lbm_ctx* c, const void* f, double* rho, double* ux, double* uz, double* T, int renorm) {
    dim3 grid((c->Lz + 127) / 128, c->Lx);
    k_moments<S><<<grid, 128, 0, c->stream>>>((const typename S::T*)f, c->Lx, c->Lz, c->grav, renorm,
                                              rho, ux, uz, T);
}

// A diagnostic's view of the current state: the state itself, or (LBM_F32_DEV) its FP64
// populations fref + d in a temporary buffer, released (stream-ordered) with the view.
struct StateView {
    const void* f = nullptr;
    int prec = LBM_F64;
    double* tmp = nullptr;
    cudaStream_t st = nullptr;
    StateView() = default;
    StateView(const StateView&) = delete;
    StateView& operator=(const StateView&) = delete;
    ~StateView() {
        if (tmp) cudaFreeAsync(tmp, st);
    }
};
static int state_view(lbm_ctx* c, StateView& v) {
    v.st = c->stream;
    if (c->prec != LBM_F32_DEV) {
        v.f = c->buf[c->cur];
        v.prec = c->prec;
        return LBM_OK;
    }
    const long long n = (long long)Q * c->Lx * c->Lz;
    if (dev_malloc_async(&v.tmp, n * sizeof(double), c->stream) != cudaSuccess)
        return fail(LBM_ENOMEM, "cannot allocate the FP64 view of the state (%lld doubles)", n);
    k_to_f64_dev<<<(unsigned int)((n + 255) / 256), 256, 0, c->stream>>>((const float*)c->buf[c->cur], 0, n,
                                                                      c->Lx * c->Lz, c->Lz, c->fref, v.tmp);
    LAUNCH_CHECK();
    v.f = v.tmp;
    v.prec = LBM_F64;
    return LBM_OK;
}

// Host equilibrium (closed form of the 4th-order Hermite expansion, long double) with the
// library's quadrature: f[l] = w_l rho P(s, |u|^2, T - 1).
static void feq_host(long double rho, long double ux, long double uz, long double T, long double (&f)[Q]) {
    const long double r = g_quad.r, r2 = r * r, th = T - 1.0L, u2 = ux * ux + uz * uz;
    for (int l = 0; l < Q; l++) {
        const long double C2 = r2 * c2(l);
        const long double s = r * (cx(l) * ux + cz(l) * uz);
        const long double K0 = 1.0L - 0.5L * u2 + 0.5L * th * (C2 - 2.0L) + 0.125L * u2 * u2
                             - 0.25L * th * u2 * (C2 - 4.0L) + 0.125L * th * th * (C2 * C2 - 8.0L * C2 + 8.0L);
        const long double K1 = 1.0L - 0.5L * u2 + 0.5L * th * (C2 - 4.0L);
        const long double K2 = 0.5L - 0.25L * u2 + 0.25L * th * (C2 - 6.0L);
        const long double P = K0 + s * (K1 + s * (K2 + s * (1.0L / 6.0L + s / 24.0L)));
        f[l] = (long double)g_quad.w_shell[shell_of(l)] * rho * P;
    }
}

// LBM_F32_DEV: build the reference of rows with means rho0[z], T0[z] (host, long double) and
// upload fref (FP64), dref and the per-row constants (FP32); see step_f32dev.cuh.  Blocks the
// host until the copies are done.
static int dev_reference(lbm_ctx* c, const double* rho0, const double* T0) {
    const int Lz = c->Lz;
    const long double r = g_quad.r, u0z = -0.5L * c->grav;
    std::vector<long double> fr((size_t)Q * Lz);
    for (int z = 0; z < Lz; z++) {
        long double f[Q];
        feq_host(rho0[z], 0.0L, u0z, T0[z], f);
        for (int l = 0; l < Q; l++) fr[(size_t)l * Lz + z] = f[l];
    }
    std::vector<double> h_fref((size_t)Q * Lz);
    std::vector<float> h_dref((size_t)NDREF * Lz), h_rowc((size_t)RC_N * Lz);
    for (int z = 0; z < Lz; z++) {
        long double R = 0, Jx = 0, Jz = 0, E = 0;
        for (int l = 0; l < Q; l++) {
            int ls = l, zs = z - cz(l);       // the pull source of population l at row z
            if (zs < 0) { ls = opp(l); zs = cz(l) - 1 - z; }
            else if (zs >= Lz) { ls = opp(l); zs = 2 * Lz - 1 - z + cz(l); }
            const long double g = fr[(size_t)ls * Lz + zs];
            h_fref[(size_t)l * Lz + z] = (double)fr[(size_t)l * Lz + z];
            if (dref_slot(l) >= 0) h_dref[(size_t)dref_slot(l) * Lz + z] = (float)(g - fr[(size_t)l * Lz + z]);
            R += g;
            Jx += cx(l) * g;
            Jz += cz(l) * g;
            E += c2(l) * g;
        }
        const long double eg = E / R, ugx = r * Jx / R, ugz = r * Jz / R, ug2 = ugx * ugx + ugz * ugz;
        const long double Tg = 0.5L * (r * r * eg - ug2);
        const float v[RC_N] = {(float)rho0[z], (float)((long double)T0[z] - 1.0L), (float)(R - rho0[z]),
                               (float)(Tg - T0[z]), (float)eg, (float)Jx, (float)Jz, (float)ug2};
        for (int k = 0; k < RC_N; k++) h_rowc[(size_t)z * RC_N + k] = v[k];
    }
    CU(cudaStreamSynchronize(c->stream));     // no step may read the tables while they change
    CU(cudaMemcpy(c->fref, h_fref.data(), h_fref.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->dref, h_dref.data(), h_dref.size() * sizeof(float), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->rowc, h_rowc.data(), h_rowc.size() * sizeof(float), cudaMemcpyHostToDevice));
    return LBM_OK;
}

extern "C" {

const char* lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_test_oob_count(unsigned int* out) {
#ifdef LBM_BOUNDS_CHECK
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpyFromSymbol(out, g_oob_count, sizeof(unsigned int)));
    const unsigned int zero = 0;
    CU(cudaMemcpyToSymbol(g_oob_count, &zero, sizeof zero));
    return LBM_OK;
#else
    (void)out;
    return fail(LBM_ESTATE, "not a bounds-checked build");
#endif
}

int lbm_test_fail_alloc(int n) {
    g_fail_alloc.store(n < 0 ? -1 : n);
    return LBM_OK;
}

int lbm_test_packed_ff(int n, unsigned long long seed, unsigned long long* mismatches) {
    if (n < 1 || !mismatches) return fail(LBM_EINVAL, "n = %d, mismatches %p", n, (void*)mismatches);
    unsigned long long* d = nullptr;
    if (dev_malloc(&d, sizeof *d) != cudaSuccess) return fail(LBM_ENOMEM, "cannot allocate the mismatch count");
    cudaError_t e = cudaMemset(d, 0, sizeof *d);
    if (e == cudaSuccess) {
        k_selftest_ffx2<<<std::min((n + 255) / 256, 4096), 256>>>(n, seed, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(mismatches, d, sizeof *d, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "packed float-float self-test: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_probe_fp64_rate(int iters, double* fma_per_s) {
    if (iters < 1 || iters > (1 << 18) || !fma_per_s)
        return fail(LBM_EINVAL, "iters = %d (1 .. 2^18), fma_per_s %p", iters, (void*)fma_per_s);
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double* d = nullptr;
    if (dev_malloc(&d, sizeof *d) != cudaSuccess) return fail(LBM_ENOMEM, "cannot allocate the probe's word");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    float ms = 0.0f;
    if (e == cudaSuccess) {
        k_probe_dfma<<<blocks, PROBE_THREADS>>>(iters, 0.999999, 1e-6, d);    // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0);
    if (e == cudaSuccess) {
        k_probe_dfma<<<blocks, PROBE_THREADS>>>(iters, 0.999999, 1e-6, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "FP64 probe: %s", cudaGetErrorString(e));
    if (!(ms > 0.0f)) return fail(LBM_ECUDA, "FP64 probe: no elapsed time");
    *fma_per_s = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters / (ms * 1e-3);
    return LBM_OK;
}

int lbm_lattice(int* c, double* w, double* r) {
    Quadrature q;
    int rc = host_quadrature(&q);
    if (rc) return rc;
    for (int l = 0; l < Q; l++) {
        if (c) { c[2 * l] = cx(l); c[2 * l + 1] = cz(l); }
        if (w) w[l] = q.w_shell[shell_of(l)];
    }
    if (r) *r = q.r;
    return LBM_OK;
}

int lbm_create(lbm_ctx** out, int Lx, int Lz, int prec, double tau, double g, void* buf0, void* buf1,
               size_t bytes, void* cuda_stream) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (Lx < 1 || Lz < 6) return fail(LBM_EINVAL, "lattice %d x %d: need Lx >= 1, Lz >= 6", Lx, Lz);
    if ((long long)Q * Lx * Lz >= (1LL << 31))
        return fail(LBM_EINVAL, "lattice %d x %d too large: 37*Lx*Lz must be < 2^31", Lx, Lz);
    if (!valid_prec(prec)) return fail(LBM_EINVAL, "unknown precision %d", prec);
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(LBM_EINVAL, "tau = %g must be > 0.5", tau);
    if (!(g >= 0.0) || !std::isfinite(g)) return fail(LBM_EINVAL, "g = %g must be >= 0", g);
    if (!buf0 || !buf1 || buf0 == buf1) return fail(LBM_EINVAL, "need two distinct device buffers");
    const size_t need = (size_t)Q * Lx * Lz * pop_bytes(prec);
    if (bytes < need) return fail(LBM_EINVAL, "buffers of %zu bytes, need %zu", bytes, need);
    if (((uintptr_t)buf0 | (uintptr_t)buf1) & 15) return fail(LBM_EINVAL, "buffers must be 16-byte aligned");
    cudaPointerAttributes a0, a1;
    CU(cudaPointerGetAttributes(&a0, buf0));
    CU(cudaPointerGetAttributes(&a1, buf1));
    if (a0.type != cudaMemoryTypeDevice || a1.type != cudaMemoryTypeDevice || a0.device != a1.device)
        return fail(LBM_EINVAL, "buffers must be device memory on one device");
    DeviceGuard dg(a0.device);
    if (!dg.ok) return fail(LBM_ECUDA, "cannot select device %d", a0.device);
    int rc = upload_lattice(a0.device);
    if (rc) return rc;
    lbm_ctx* c = new lbm_ctx();
    c->Lx = Lx; c->Lz = Lz; c->prec = prec; c->tau = tau; c->grav = g;
    c->buf[0] = buf0; c->buf[1] = buf1; c->bytes = bytes; c->cur = 0;
    c->stream = (cudaStream_t)cuda_stream;
    c->device = a0.device;
    bool ok = dev_malloc(&c->zcol, 2 * (size_t)Lx * sizeof(double)) == cudaSuccess &&
              dev_malloc(&c->small, ((size_t)Lz + 8) * sizeof(double)) == cudaSuccess &&
              dev_malloc(&c->dLrow, (size_t)Lz * sizeof(double)) == cudaSuccess &&
              dev_malloc(&c->colred, 2 * (size_t)Lx * sizeof(double)) == cudaSuccess &&
              dev_malloc(&c->err, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        free_ctx(c);
        return fail(LBM_ENOMEM, "context scratch allocation failed");
    }
    if (cudaMemset(c->err, 0, sizeof(unsigned int)) != cudaSuccess) {
        free_ctx(c);
        return fail(LBM_ECUDA, "memset of the error word failed");
    }
    if (prec == LBM_F32_DEV) {     // the reference of a uniform state until lbm_init_layers
        ok = dev_malloc(&c->fref, (size_t)Q * Lz * sizeof(double)) == cudaSuccess &&
             dev_malloc(&c->dref, (size_t)NDREF * Lz * sizeof(float)) == cudaSuccess &&
             dev_malloc(&c->rowc, (size_t)RC_N * Lz * sizeof(float)) == cudaSuccess;
        if (!ok) {
            free_ctx(c);
            return fail(LBM_ENOMEM, "reference table allocation failed");
        }
        const std::vector<double> one((size_t)Lz, 1.0);
        rc = dev_reference(c, one.data(), one.data());
        if (rc) {
            free_ctx(c);
            return rc;
        }
    }
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_OK;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return LBM_OK;
}

void* lbm_current(lbm_ctx* c) { return c ? c->buf[c->cur] : nullptr; }

int lbm_sync(lbm_ctx* c) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    DeviceGuard dg(c->device);
    CU(cudaStreamSynchronize(c->stream));
    unsigned int e = 0;
    CU(cudaMemcpy(&e, c->err, sizeof e, cudaMemcpyDeviceToHost));
    if (e) {
        CU(cudaMemset(c->err, 0, sizeof e));
        return fail(LBM_ETIMEOUT, "device error word 0x%x (bounded wait gave up)", e);
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// Init
// ---------------------------------------------------------------------------------
static int fill_init_params(lbm_ctx* c, const lbm_layers_desc* d, InitParams* ip) {
    if (!d) return fail(LBM_EINVAL, "layers desc is NULL");
    if (!(d->T_u > 0 && d->T_m > 0 && d->T_d > 0)) return fail(LBM_EINVAL, "temperatures must be > 0");
    if (!(d->tanh_w > 0)) return fail(LBM_EINVAL, "tanh_w must be > 0");
    if (!(d->rho_ref > 0)) return fail(LBM_EINVAL, "rho_ref must be > 0");
    if (d->n_modes < 0) return fail(LBM_EINVAL, "n_modes < 0");
    if (d->n_modes > 0 && (!d->amp_lo || !d->phase_lo || !d->amp_hi || !d->phase_hi))
        return fail(LBM_EINVAL, "mode arrays are NULL");
    ip->Lx = c->Lx; ip->Lz = c->Lz; ip->plane = c->Lx * c->Lz;
    ip->grav = c->grav; ip->Tu = d->T_u; ip->Tm = d->T_m; ip->Td = d->T_d;
    ip->rho_ref = d->rho_ref; ip->wt = d->tanh_w; ip->zlo0 = d->z_lo; ip->zhi0 = d->z_hi;
    ip->K = d->n_modes;
    const int cap = std::max(1, d->n_modes);
    if (c->modes_cap < cap) {
        if (c->modes) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->modes);
        }
        c->modes = nullptr;
        c->modes_cap = 0;
        if (dev_malloc(&c->modes, 4 * (size_t)cap * sizeof(double)) != cudaSuccess)
            return fail(LBM_ENOMEM, "mode buffer allocation failed");
        c->modes_cap = cap;
    }
    if (d->n_modes > 0) {
        std::vector<double> h(4 * (size_t)d->n_modes);
        for (int k = 0; k < d->n_modes; k++) {
            h[k] = d->amp_lo[k];
            h[d->n_modes + k] = d->phase_lo[k];
            h[2 * d->n_modes + k] = d->amp_hi[k];
            h[3 * d->n_modes + k] = d->phase_hi[k];
        }
        CU(cudaMemcpyAsync(c->modes, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CU(cudaStreamSynchronize(c->stream));   // h is released at scope exit
    }
    return LBM_OK;
}

int lbm_init_layers(lbm_ctx* c, const lbm_layers_desc* d) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    DeviceGuard dg(c->device);
    InitParams ip;
    int rc = fill_init_params(c, d, &ip);
    if (rc) return rc;
    k_interfaces<<<(c->Lx + 127) / 128, 128, 0, c->stream>>>(c->zcol, c->modes, ip);
    LAUNCH_CHECK();
    dim3 grid((c->Lz + 127) / 128, c->Lx);
    void* f = c->buf[c->cur];
    if (c->prec == LBM_F32_DEV) {      // reference of the initial rows, then the deviations
        rc = ensure_part(c, 2 * (size_t)c->Lz);
        if (rc) return rc;
        k_init_rowmeans<<<c->Lz, 128, 0, c->stream>>>(c->zcol, ip, c->part);
        LAUNCH_CHECK();
        std::vector<double> h(2 * (size_t)c->Lz);
        CU(cudaMemcpyAsync(h.data(), c->part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        rc = dev_reference(c, h.data(), h.data() + c->Lz);
        if (rc) return rc;
        k_init_dev<<<grid, 128, 0, c->stream>>>((float*)f, c->zcol, ip, c->fref);
        LAUNCH_CHECK();
        return LBM_OK;
    }
    switch (c->prec) {
        case LBM_F64:
        case LBM_F64_FF:
            k_init<StoreF64><<<grid, 128, 0, c->stream>>>((double*)f, c->zcol, ip);
            break;
        default:
            k_init<StoreF32><<<grid, 128, 0, c->stream>>>((float*)f, c->zcol, ip);
            break;
    }
    LAUNCH_CHECK();
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// Step
// ---------------------------------------------------------------------------------
int lbm_set_walls(lbm_ctx* c, int thermal, double T_bottom, double T_top) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (thermal != 0 && thermal != 1) return fail(LBM_EINVAL, "thermal must be 0 or 1");
    if (thermal && !(T_bottom > 0.0 && T_top > 0.0 && std::isfinite(T_bottom) && std::isfinite(T_top)))
        return fail(LBM_EINVAL, "wall temperatures must be positive and finite");
    if (thermal) NOT_DEV(c, "the thermal wall rule");
    if (thermal) {
        thermal_wall_q(quad_w_shell(), g_quad.r, T_bottom, 0, c->tw.q[0]);
        thermal_wall_q(quad_w_shell(), g_quad.r, T_top, 1, c->tw.q[1]);
    }
    c->thermal = thermal;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int nsteps) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
    DeviceGuard dg(c->device);
    const StepParams p = step_params(c);
    for (int s = 0; s < nsteps; s++) {
        ctx_step(c, c->buf[c->cur], c->buf[c->cur ^ 1], p, c->stream);
        LAUNCH_CHECK();
        c->cur ^= 1;
    }
    return LBM_OK;
}

int lbm_step_push(lbm_ctx* c, int nsteps) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
    NEED_BOUNCE_BACK(c, "lbm_step_push");
    NOT_DEV(c, "lbm_step_push");
    DeviceGuard dg(c->device);
    const StepParams p = step_params(c);
    const Tiling t = make_tiling(p.Lx, p.Lz, BLOCK_Z);
    for (int s = 0; s < nsteps; s++) {
        const void* fin = c->buf[c->cur];
        void* fout = c->buf[c->cur ^ 1];
        switch (c->prec) {
            case LBM_F64: launch_step_f64_push((const double*)fin, (double*)fout, p, t, c->stream); break;
            case LBM_F64_FF:
                launch_step_ff_push((const double*)fin, (double*)fout, p, quad_w_shell(), t, c->stream);
                break;
            default: launch_step_f32_push((const float*)fin, (float*)fout, p, t, c->stream); break;
        }
        LAUNCH_CHECK();
        c->cur ^= 1;
    }
    return LBM_OK;
}

int lbm_step_chain(lbm_ctx* c, void* const* states, int n) {
    if (!c || !states) return fail(LBM_EINVAL, "NULL argument");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    for (int j = 0; j < n; j++) {
        if (!states[j]) return fail(LBM_EINVAL, "state %d is NULL", j);
        if (j > 0 && states[j] == states[j - 1]) return fail(LBM_EINVAL, "states %d and %d are the same buffer", j - 1, j);
    }
    DeviceGuard dg(c->device);
    const StepParams p = step_params(c);
    for (int j = 0; j + 1 < n; j++) {
        ctx_step(c, states[j], states[j + 1], p, c->stream);
        LAUNCH_CHECK();
    }
    return LBM_OK;
}

int lbm_propagate(lbm_ctx* c) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    NOT_DEV(c, "lbm_propagate");
    DeviceGuard dg(c->device);
    const Tiling t = make_tiling(c->Lx, c->Lz, BLOCK_Z);
    const void* fin = c->buf[c->cur];
    void* fout = c->buf[c->cur ^ 1];
    if (pop_bytes(c->prec) == 8)
        k_propagate<double><<<tiling_blocks(t), BLOCK_Z, 0, c->stream>>>((const double*)fin, (double*)fout, c->Lx, c->Lz, t);
    else
        k_propagate<float><<<tiling_blocks(t), BLOCK_Z, 0, c->stream>>>((const float*)fin, (float*)fout, c->Lx, c->Lz, t);
    LAUNCH_CHECK();
    c->cur ^= 1;
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// Population copies
// ---------------------------------------------------------------------------------
static int convert_pops(lbm_ctx* c, double* buf, int on_device, bool to_f64) {
    const long long n = (long long)Q * c->Lx * c->Lz;
    void* f = c->buf[c->cur];
    if (c->prec == LBM_F64 || c->prec == LBM_F64_FF) {
        cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice
                                     : (to_f64 ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
        if (to_f64) CU(cudaMemcpyAsync(buf, f, n * sizeof(double), k, c->stream));
        else CU(cudaMemcpyAsync(f, buf, n * sizeof(double), k, c->stream));
        if (!on_device) CU(cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    // FP32 storage: convert one population plane at a time through device scratch
    const long long chunk = (long long)c->Lx * c->Lz;
    double* tmp = nullptr;
    if (!on_device && dev_malloc_async(&tmp, chunk * sizeof(double), c->stream) != cudaSuccess)
        return fail(LBM_ENOMEM, "conversion buffer allocation failed");
    for (long long first = 0; first < n; first += chunk) {
        const long long m = std::min(chunk, n - first);
        double* dev = on_device ? buf + first : tmp;
        const int blocks = (int)((m + 255) / 256);
        if (to_f64) {
            if (c->prec == LBM_F32_DEV)
                k_to_f64_dev<<<blocks, 256, 0, c->stream>>>((const float*)f, first, m, (int)chunk, c->Lz, c->fref, dev);
            else
                k_to_f64<StoreF32><<<blocks, 256, 0, c->stream>>>((float*)f, first, m, dev);
            LAUNCH_CHECK();
            if (!on_device) CU(cudaMemcpyAsync(buf + first, tmp, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        } else {
            if (!on_device) CU(cudaMemcpyAsync(tmp, buf + first, m * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            if (c->prec == LBM_F32_DEV)
                k_from_f64_dev<<<blocks, 256, 0, c->stream>>>((float*)f, first, m, (int)chunk, c->Lz, c->fref, dev);
            else
                k_from_f64<StoreF32><<<blocks, 256, 0, c->stream>>>((float*)f, first, m, dev);
            LAUNCH_CHECK();
        }
        if (!on_device) CU(cudaStreamSynchronize(c->stream));
    }
    if (tmp) {
        CU(cudaFreeAsync(tmp, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* f, int on_device) {
    if (!c || !f) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(c->device);
    return convert_pops(c, f, on_device, true);
}

int lbm_set_populations(lbm_ctx* c, const double* f, int on_device) {
    if (!c || !f) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(c->device);
    return convert_pops(c, const_cast<double*>(f), on_device, false);
}

int lbm_step_host(lbm_ctx* c, const double* const* host_in, double* const* host_out, int n) {
    if (!c || !host_in || !host_out) return fail(LBM_EINVAL, "NULL argument");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    if (pop_bytes(c->prec) != 8) return fail(LBM_EINVAL, "lbm_step_host needs FP64 storage");
    for (int t = 0; t < n; t++)
        if (!host_in[t] || !host_out[t]) return fail(LBM_EINVAL, "host buffer %d is NULL", t);
    DeviceGuard dg(c->device);
    constexpr int NCOPY = 2;          // copy streams per direction
    if (!c->e_step) {                  // first use: all streams and events, or none
        cudaStream_t si[NCOPY] = {}, so[NCOPY] = {};
        cudaEvent_t ei[NCOPY] = {}, eo[NCOPY] = {}, es = nullptr;
        bool ok = cudaEventCreateWithFlags(&es, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < NCOPY; k++)
            ok = cudaStreamCreateWithFlags(&si[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&so[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ei[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&eo[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            for (int k = 0; k < NCOPY; k++) {
                if (si[k]) cudaStreamDestroy(si[k]);
                if (so[k]) cudaStreamDestroy(so[k]);
                if (ei[k]) cudaEventDestroy(ei[k]);
                if (eo[k]) cudaEventDestroy(eo[k]);
            }
            if (es) cudaEventDestroy(es);
            return fail(LBM_ECUDA, "copy streams could not be created");
        }
        for (int k = 0; k < NCOPY; k++) {
            c->s_in[k] = si[k];
            c->s_out[k] = so[k];
            c->e_in[k] = ei[k];
            c->e_out[k] = eo[k];
        }
        c->e_step = es;
    }
    const size_t bytes = (size_t)Q * c->Lx * c->Lz * sizeof(double);
    size_t off[NCOPY + 1];            // the state in NCOPY parts of whole populations
    for (int k = 0; k <= NCOPY; k++) off[k] = (size_t)((Q * k) / NCOPY) * (bytes / Q);
    const StepParams p = step_params(c);
    char* X = (char*)c->buf[c->cur];         // the step's input, filled from the host
    char* Y = (char*)c->buf[c->cur ^ 1];     // the step's output, read back to the host
    // Step t: X <- host_in[t] (s_in), Y = step(X) (c's stream), host_out[t] <- Y (s_out).
    // The copy in of step t waits until step t-1 has read X; the step waits for its copy
    // in and for the copy out of step t-1 to have read Y.  So the copy out of step t-1
    // and the copy in of step t run at the same time, one per direction of the link; each
    // is split over NCOPY streams (one stream per direction left the host-to-device copy at
    // ~40 GB/s when it ran alone, two reach ~54).
    CU(cudaEventRecord(c->e_step, c->stream));
    for (int k = 0; k < NCOPY; k++) CU(cudaEventRecord(c->e_out[k], c->stream));
    for (int t = 0; t < n; t++) {
        for (int k = 0; k < NCOPY; k++) {
            CU(cudaStreamWaitEvent(c->s_in[k], c->e_step, 0));
            CU(cudaMemcpyAsync(X + off[k], (const char*)host_in[t] + off[k], off[k + 1] - off[k],
                               cudaMemcpyHostToDevice, c->s_in[k]));
            CU(cudaEventRecord(c->e_in[k], c->s_in[k]));
            CU(cudaStreamWaitEvent(c->stream, c->e_in[k], 0));
            CU(cudaStreamWaitEvent(c->stream, c->e_out[k], 0));
        }
        ctx_step(c, X, Y, p, c->stream);
        LAUNCH_CHECK();
        CU(cudaEventRecord(c->e_step, c->stream));
        for (int k = 0; k < NCOPY; k++) {
            CU(cudaStreamWaitEvent(c->s_out[k], c->e_step, 0));
            CU(cudaMemcpyAsync((char*)host_out[t] + off[k], Y + off[k], off[k + 1] - off[k],
                               cudaMemcpyDeviceToHost, c->s_out[k]));
            CU(cudaEventRecord(c->e_out[k], c->s_out[k]));
        }
    }
    for (int k = 0; k < NCOPY; k++) {
        CU(cudaStreamSynchronize(c->s_in[k]));
        CU(cudaStreamSynchronize(c->s_out[k]));
    }
    CU(cudaStreamSynchronize(c->stream));
    if (n > 0) c->cur ^= 1;           // the device now holds the last step's output
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// Diagnostics
// ---------------------------------------------------------------------------------
int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uz, double* T, int renormalised, int on_device) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    DeviceGuard dg(c->device);
    const size_t n = (size_t)c->Lx * c->Lz;
    double* outs[4] = {rho, ux, uz, T};
    double* dev[4] = {rho, ux, uz, T};
    double* tmp = nullptr;
    if (!on_device) {
        int k = 0;
        for (int i = 0; i < 4; i++) k += outs[i] != nullptr;
        if (k == 0) return LBM_OK;
        if (dev_malloc_async(&tmp, k * n * sizeof(double), c->stream) != cudaSuccess)
            return fail(LBM_ENOMEM, "moments buffer allocation failed");
        k = 0;
        for (int i = 0; i < 4; i++) dev[i] = outs[i] ? tmp + (k++) * n : nullptr;
    }
    StateView v;
    int rc = state_view(c, v);
    if (rc) {
        if (tmp) cudaFreeAsync(tmp, c->stream);
        return rc;
    }
    switch (v.prec) {
        case LBM_F64: case LBM_F64_FF: launch_moments<StoreF64>(c, v.f, dev[0], dev[1], dev[2], dev[3], renormalised); break;
        default: launch_moments<StoreF32>(c, v.f, dev[0], dev[1], dev[2], dev[3], renormalised); break;
    }
    LAUNCH_CHECK();
    if (!on_device) {
        for (int i = 0; i < 4; i++)
            if (outs[i]) CU(cudaMemcpyAsync(outs[i], dev[i], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaFreeAsync(tmp, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

static int row_mean_device(lbm_ctx* c, double* Tbar_dev) {
    const int target = std::max(1, (148 * 16 * 128) / std::max(1, c->Lz));
    const int nx_per = (c->Lx + std::min(c->Lx, target) - 1) / std::min(c->Lx, target);
    const int nch = (c->Lx + nx_per - 1) / nx_per;
    int rc = ensure_part(c, (size_t)nch * c->Lz);
    if (rc) return rc;
    dim3 grid((c->Lz + 127) / 128, nch);
    StateView v;
    rc = state_view(c, v);
    if (rc) return rc;
    const void* f = v.f;
    const int part_n = (int)std::min(c->part_cap, (size_t)INT_MAX);
    switch (v.prec) {
        case LBM_F64: case LBM_F64_FF:
            k_rowT_partial<StoreF64><<<grid, 128, 0, c->stream>>>((const double*)f, c->Lx, c->Lz, nx_per, c->part, part_n); break;
        default:
            k_rowT_partial<StoreF32><<<grid, 128, 0, c->stream>>>((const float*)f, c->Lx, c->Lz, nx_per, c->part, part_n); break;
    }
    LAUNCH_CHECK();
    k_rowT_final<<<(c->Lz + 127) / 128, 128, 0, c->stream>>>(c->part, part_n, nch, c->Lx, c->Lz, Tbar_dev);
    LAUNCH_CHECK();
    return LBM_OK;
}

int lbm_row_mean_T(lbm_ctx* c, double* Tbar, int on_device) {
    if (!c || !Tbar) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(c->device);
    double* dst = on_device ? Tbar : c->small;
    int rc = row_mean_device(c, dst);
    if (rc) return rc;
    if (!on_device) {
        CU(cudaMemcpyAsync(Tbar, c->small, (size_t)c->Lz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_tent_widths(lbm_ctx* c, double T_u, double T_m, double T_d, double out[2]) {
    if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
    if (!(T_u < T_m && T_m < T_d)) return fail(LBM_EINVAL, "need T_u < T_m < T_d");
    DeviceGuard dg(c->device);
    int rc = row_mean_device(c, c->small);
    if (rc) return rc;
    double* res = c->small + c->Lz;
    k_tent_widths<<<1, 256, 0, c->stream>>>(c->small, c->Lz, T_u, T_m, T_d, res);
    LAUNCH_CHECK();
    CU(cudaMemcpyAsync(out, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_row_stats(lbm_ctx* c, double* T_mean, double* T_rms, double* Ek_mean, double* Ek_rms, int on_device) {
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    if (!T_mean && !T_rms && !Ek_mean && !Ek_rms) return LBM_OK;
    DeviceGuard dg(c->device);
    const int Lz = c->Lz;
    const int target = std::max(1, (148 * 16 * 128) / std::max(1, Lz));
    const int nx_per = (c->Lx + std::min(c->Lx, target) - 1) / std::min(c->Lx, target);
    const int nch = (c->Lx + nx_per - 1) / nx_per;
    // part: 2 * nch * Lz partial sums, then 4 * Lz results (means, rms)
    int rc = ensure_part(c, (size_t)(2 * nch + 4) * Lz);
    if (rc) return rc;
    double* means = c->part + (size_t)2 * nch * Lz;
    double* rms = means + 2 * (size_t)Lz;
    dim3 grid((Lz + 127) / 128, nch);
    StateView v;
    rc = state_view(c, v);
    if (rc) return rc;
    const void* f = v.f;
    for (int pass = 0; pass < 2; pass++) {
        const double* m = pass ? means : nullptr;
        switch (v.prec) {
            case LBM_F64: case LBM_F64_FF:
                k_row_stats_partial<StoreF64><<<grid, 128, 0, c->stream>>>((const double*)f, c->Lx, Lz, nx_per, c->grav, m, c->part);
                break;
            default:
                k_row_stats_partial<StoreF32><<<grid, 128, 0, c->stream>>>((const float*)f, c->Lx, Lz, nx_per, c->grav, m, c->part);
                break;
        }
        LAUNCH_CHECK();
        k_row_stats_final<<<(Lz + 127) / 128, 128, 0, c->stream>>>(c->part, nch, c->Lx, Lz, pass, pass ? rms : means);
        LAUNCH_CHECK();
    }
    const double* src[4] = {means, rms, means + Lz, rms + Lz};
    double* dst[4] = {T_mean, T_rms, Ek_mean, Ek_rms};
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int i = 0; i < 4; i++)
        if (dst[i]) CU(cudaMemcpyAsync(dst[i], src[i], (size_t)Lz * sizeof(double), kind, c->stream));
    if (!on_device) CU(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_widths(lbm_ctx* c, double T_u, double T_m, double T_d, double out[2], double* dL_dTbar) {
    if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
    if (!(T_u < T_m && T_m < T_d)) return fail(LBM_EINVAL, "need T_u < T_m < T_d");
    DeviceGuard dg(c->device);
    int rc = row_mean_device(c, c->small);
    if (rc) return rc;
    double* res = c->small + c->Lz;   // 3 doubles after Tbar
    k_widths<<<1, 32, 0, c->stream>>>(c->small, c->Lz, T_u, T_m, T_d, res, dL_dTbar ? c->dLrow : nullptr);
    LAUNCH_CHECK();
    double h[3];
    CU(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    if (dL_dTbar) CU(cudaMemcpyAsync(dL_dTbar, c->dLrow, (size_t)c->Lz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h[2] != 0.0) return fail(LBM_EINVAL, "a mixing-width crossing is missing");
    out[0] = h[0];
    out[1] = h[1];
    return LBM_OK;
}

int lbm_global_sums(lbm_ctx* c, double out[2]) {
    if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
    DeviceGuard dg(c->device);
    const int nsite = c->Lx * c->Lz;
    const int nblk = std::max(1, std::min(148 * 8, (nsite + RED_THREADS - 1) / RED_THREADS));
    int rc = ensure_part(c, 2 * (size_t)nblk);
    if (rc) return rc;
    StateView v;
    rc = state_view(c, v);
    if (rc) return rc;
    const void* f = v.f;
    switch (v.prec) {
        case LBM_F64: case LBM_F64_FF:
            k_global_partial<StoreF64><<<nblk, RED_THREADS, 0, c->stream>>>((const double*)f, c->Lx, c->Lz, c->part); break;
        default:
            k_global_partial<StoreF32><<<nblk, RED_THREADS, 0, c->stream>>>((const float*)f, c->Lx, c->Lz, c->part); break;
    }
    LAUNCH_CHECK();
    k_global_final<<<1, RED_THREADS, 0, c->stream>>>(c->part, nblk, c->small);
    LAUNCH_CHECK();
    CU(cudaMemcpyAsync(out, c->small, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return fail(LBM_ENUMERIC, "non-finite mass or energy");
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------------
// Buffers in the context's storage precision (double for LBM_F64 / LBM_F64_FF, float for LBM_F32).
static void launch_adjoint(const lbm_ctx* c, const void* f_t, const void* lam_next, void* lam_out,
                           const StepParams& p) {
    const double *fd = (const double*)f_t, *ld = (const double*)lam_next;
    double* od = (double*)lam_out;
    dim3 grid((c->Lz + BLOCK_Z - 1) / BLOCK_Z, c->Lx);
    if (c->thermal) {               // LBM_F64_FF with its ghost scratch (adjoint_walls_ready)
        launch_adjoint_ff_thermal(fd, ld, od, p, quad_w_shell(), g_quad.r, c->tw, c->gmu, c->stream);
    } else if (c->prec == LBM_F64_FF) {
        launch_adjoint_ff(fd, ld, od, p, quad_w_shell(), g_quad.r, make_tiling(c->Lx, c->Lz, BLOCK_Z), c->stream);
    } else if (c->prec == LBM_F64) {
        launch_pdl(k_adjoint_native_f64, grid, BLOCK_Z, c->stream, fd, ld, od, p);
    } else {
        launch_pdl(k_adjoint_native_f32, grid, BLOCK_Z, c->stream, (const float*)f_t, (const float*)lam_next,
                   (float*)lam_out, p);
    }
}

// The adjoint with the context's wall rule can run: thermal walls need LBM_F64_FF and the
// ghost-pull scratch (allocated here on first use).
static int adjoint_walls_ready(lbm_ctx* c) {
    if (!c->thermal) return LBM_OK;
    if (c->prec != LBM_F64_FF) return fail(LBM_ESTATE, "the adjoint with thermal walls needs an LBM_F64_FF context");
    if (!c->gmu && dev_malloc(&c->gmu, (size_t)6 * Q * c->Lx * sizeof(double)) != cudaSuccess)
        return fail(LBM_ENOMEM, "thermal-wall adjoint scratch allocation failed");
    return LBM_OK;
}

int lbm_adjoint_step(lbm_ctx* c, const void* f_t, const void* lam_next, void* lam_out) {
    if (!c || !f_t || !lam_next || !lam_out) return fail(LBM_EINVAL, "NULL argument");
    if (lam_out == lam_next || lam_out == f_t) return fail(LBM_EINVAL, "lam_out must not alias the inputs");
    NOT_DEV(c, "the adjoint step");
    DeviceGuard dg(c->device);
    int rc = adjoint_walls_ready(c);
    if (rc) return rc;
    launch_adjoint(c, f_t, lam_next, lam_out, step_params(c));
    LAUNCH_CHECK();
    return LBM_OK;
}

int lbm_adjoint_chain(lbm_ctx* c, const void* const* states, int n, void* lam_a, void* lam_b, int* out_index) {
    if (!c || !states || !lam_a || !lam_b || !out_index) return fail(LBM_EINVAL, "NULL argument");
    NOT_DEV(c, "the adjoint step");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    if (lam_a == lam_b) return fail(LBM_EINVAL, "lam_a and lam_b must differ");
    for (int j = 0; j < n; j++) {
        if (!states[j]) return fail(LBM_EINVAL, "state %d is NULL", j);
        if (states[j] == lam_a || states[j] == lam_b) return fail(LBM_EINVAL, "state %d aliases an adjoint buffer", j);
    }
    DeviceGuard dg(c->device);
    int rc = adjoint_walls_ready(c);
    if (rc) return rc;
    const StepParams p = step_params(c);
    void* lam[2] = {lam_a, lam_b};
    int cur = 0;
    for (int j = n - 1; j >= 0; j--) {
        launch_adjoint(c, states[j], lam[cur], lam[cur ^ 1], p);
        LAUNCH_CHECK();
        cur ^= 1;
    }
    *out_index = cur;
    return LBM_OK;
}

int lbm_record_moments(lbm_ctx* c, const double* f0, int n, double* work_a, double* work_b,
                       int64_t* const* moments) {
    if (!c || !f0 || !work_a || !work_b || !moments) return fail(LBM_EINVAL, "NULL argument");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    if (c->prec != LBM_F64_FF) return fail(LBM_ESTATE, "moment records need an LBM_F64_FF context");
    NEED_BOUNCE_BACK(c, "the adjoint step");
    if (work_a == work_b || f0 == work_a || f0 == work_b) return fail(LBM_EINVAL, "f0, work_a, work_b must differ");
    for (int j = 0; j < n; j++)
        if (!moments[j]) return fail(LBM_EINVAL, "moment record %d is NULL", j);
    DeviceGuard dg(c->device);
    const StepParams p = step_params(c);
    const Tiling t = make_tiling(p.Lx, p.Lz, BLOCK_Z);
    const StepParamsFF q = ff_params(p, quad_w_shell());
    double* w[2] = {work_a, work_b};
    for (int j = 0; j < n; j++) {
        const double* fin = j == 0 ? f0 : w[(j - 1) & 1];
        launch_pdl(k_step_ff_moments, tiling_blocks(t), BLOCK_Z, c->stream, fin, w[j & 1], q, t, moments[j]);
        LAUNCH_CHECK();
    }
    return LBM_OK;
}

int lbm_adjoint_chain_moments(lbm_ctx* c, const int64_t* const* moments, int n, double* lam_a, double* lam_b,
                              int* out_index) {
    if (!c || !moments || !lam_a || !lam_b || !out_index) return fail(LBM_EINVAL, "NULL argument");
    if (n < 0) return fail(LBM_EINVAL, "n < 0");
    if (c->prec != LBM_F64_FF) return fail(LBM_ESTATE, "moment records need an LBM_F64_FF context");
    NEED_BOUNCE_BACK(c, "the adjoint step");
    if (lam_a == lam_b) return fail(LBM_EINVAL, "lam_a and lam_b must differ");
    for (int j = 0; j < n; j++)
        if (!moments[j]) return fail(LBM_EINVAL, "moment record %d is NULL", j);
    DeviceGuard dg(c->device);
    const StepParams p = step_params(c);
    const Tiling t = make_tiling(p.Lx, p.Lz, BLOCK_Z);
    double* lam[2] = {lam_a, lam_b};
    int cur = 0;
    for (int j = n - 1; j >= 0; j--) {
        launch_adjoint_ff_moments(moments[j], lam[cur], lam[cur ^ 1], p, quad_w_shell(), g_quad.r, t, c->stream);
        LAUNCH_CHECK();
        cur ^= 1;
    }
    *out_index = cur;
    return LBM_OK;
}

int lbm_loss_adjoint(lbm_ctx* c, const void* f, const double* dL_dTbar, void* lam_out) {
    if (!c || !f || !dL_dTbar || !lam_out) return fail(LBM_EINVAL, "NULL argument");
    NOT_DEV(c, "the loss adjoint");
    DeviceGuard dg(c->device);
    CU(cudaMemcpyAsync(c->dLrow, dL_dTbar, (size_t)c->Lz * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    dim3 grid((c->Lz + 127) / 128, c->Lx);
    if (c->prec == LBM_F32)
        k_loss_adjoint<StoreF32><<<grid, 128, 0, c->stream>>>((const float*)f, c->dLrow, (float*)lam_out, c->Lx, c->Lz);
    else
        k_loss_adjoint<StoreF64><<<grid, 128, 0, c->stream>>>((const double*)f, c->dLrow, (double*)lam_out, c->Lx,
                                                              c->Lz);
    LAUNCH_CHECK();
    CU(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_init_adjoint_full(lbm_ctx* c, const lbm_layers_desc* d, const void* lam0, double* dA_lo, double* dA_hi,
                          double* dph_lo, double* dph_hi) {
    if (!c || !lam0) return fail(LBM_EINVAL, "NULL argument");
    NOT_DEV(c, "the initial-state adjoint");
    DeviceGuard dg(c->device);
    InitParams ip;
    int rc = fill_init_params(c, d, &ip);
    if (rc) return rc;
    if (d->n_modes > 0 && (!dA_lo || !dA_hi)) return fail(LBM_EINVAL, "NULL gradient outputs");
    if ((dph_lo == nullptr) != (dph_hi == nullptr)) return fail(LBM_EINVAL, "give both phase outputs or neither");
    k_interfaces<<<(c->Lx + 127) / 128, 128, 0, c->stream>>>(c->zcol, c->modes, ip);
    LAUNCH_CHECK();
    if (c->prec == LBM_F32)
        k_init_adjoint_columns<StoreF32><<<c->Lx, 128, 0, c->stream>>>((const float*)lam0, c->zcol, ip, c->colred);
    else
        k_init_adjoint_columns<StoreF64><<<c->Lx, 128, 0, c->stream>>>((const double*)lam0, c->zcol, ip, c->colred);
    LAUNCH_CHECK();
    if (d->n_modes == 0) return lbm_sync(c);
    const int K = d->n_modes;
    rc = ensure_part(c, 4 * (size_t)K);
    if (rc) return rc;
    k_init_adjoint_modes<<<K, 128, 0, c->stream>>>(c->colred, c->modes, ip, c->part);
    LAUNCH_CHECK();
    std::vector<double> h(4 * (size_t)K);
    CU(cudaMemcpyAsync(h.data(), c->part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < K; k++) {
        dA_lo[k] = h[k];
        dA_hi[k] = h[K + k];
        if (dph_lo) {
            dph_lo[k] = h[2 * K + k];
            dph_hi[k] = h[3 * K + k];
        }
    }
    return LBM_OK;
}

int lbm_init_adjoint(lbm_ctx* c, const lbm_layers_desc* d, const void* lam0, double* dA_lo, double* dA_hi) {
    return lbm_init_adjoint_full(c, d, lam0, dA_lo, dA_hi, nullptr, nullptr);
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Ensembles of lattices (lbm_ensemble_*)
// ---------------------------------------------------------------------------------
struct lbm_ensemble {
    int n = 0, prec = 0, device = 0;
    cudaStream_t stream = nullptr;
    std::vector<lbm_ctx*> ctx;
    std::vector<EnsLattice> h_lats;
    EnsLattice* d_lats = nullptr;
    int total_tiles = 0;
    int total_items = 0;     // persistent work items per step
    EnsControl* d_ctl = nullptr;
    unsigned int* d_done = nullptr;
    int mode = 1;            // 0: one launch per step, 1: one persistent launch
    int tz = 128;            // tile height (threads per CTA)
    int ctas_per_sm = 0;     // persistent grid: CTAs per SM (0: as many as fit)
    long long spin_limit = 4000000000LL;   // cycles (~2 s at 2 GHz)
    unsigned int extra_wait = 0;
    cudaGraphExec_t gexec = nullptr;
    std::vector<int> g_cur;
    int g_steps = 0;
};

static int ens_layout(lbm_ensemble* e) {
    e->h_lats.resize(e->n);
    int tb = 0, ib = 0;
    for (int i = 0; i < e->n; i++) {
        lbm_ctx* c = e->ctx[i];
        NEED_BOUNCE_BACK(c, "an ensemble");
        EnsLattice& L = e->h_lats[i];
        L.buf[0] = c->buf[0];
        L.buf[1] = c->buf[1];
        L.Lx = c->Lx; L.Lz = c->Lz; L.plane = c->Lx * c->Lz;
        L.cur = c->cur;
        L.t = make_tiling(c->Lx, c->Lz, e->tz);
        L.tile_begin = tb;
        L.ntiles = tiling_blocks(L.t);
        L.item_begin = ib;
        tb += L.ntiles;
        ib += ens_items(e->prec == LBM_F64_FF, L.t.nwall, L.ntiles);
    }
    e->total_tiles = tb;
    e->total_items = ib;
    // stream-ordered: kernels of an earlier call on the same stream still read the old table
    // (a pageable source is staged before the call returns, so h_lats may change afterwards)
    CU(cudaMemcpyAsync(e->d_lats, e->h_lats.data(), e->n * sizeof(EnsLattice), cudaMemcpyHostToDevice,
                       e->stream));
    return LBM_OK;
}

template <class P, int TZ>
static int ens_launch_tz(lbm_ensemble* e, const P& q, int nsteps) {
    if (e->mode == 0) {
        for (int s = 0; s < nsteps; s++) {
            k_ens_step<P, TZ><<<e->total_tiles, TZ, 0, e->stream>>>(e->d_lats, e->n, q, s);
            LAUNCH_CHECK();
        }
        return LBM_OK;
    }
    if ((long long)nsteps * e->total_items >= (1LL << 32)) return fail(LBM_EINVAL, "too many work items for one launch");
    int per_sm = 0, nsm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<P, TZ>, TZ, 0));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, e->device));
    if (per_sm < 1) return fail(LBM_ECUDA, "persistent ensemble kernel does not fit on an SM");
    if (e->ctas_per_sm > 0) per_sm = std::min(per_sm, e->ctas_per_sm);
    CU(cudaMemsetAsync(e->d_ctl, 0, sizeof(EnsControl), e->stream));
    CU(cudaMemsetAsync(e->d_done, 0, e->n * sizeof(unsigned int), e->stream));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(per_sm * nsm);
    cfg.blockDim = dim3(TZ);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CU(cudaLaunchKernelEx(&cfg, k_ens_persistent<P, TZ>, (const EnsLattice*)e->d_lats, e->n, q, nsteps,
                          e->total_items, e->d_ctl, e->d_done, e->spin_limit, e->extra_wait));
    return LBM_OK;
}

static int ens_launch(lbm_ensemble* e, int nsteps) {
    lbm_ctx* c0 = e->ctx[0];
    const StepParams p = step_params(c0);
    if (e->prec == LBM_F64_FF) {
        const StepParamsFF q = ff_params(p, quad_w_shell());
        switch (e->tz) {
            case 64: return ens_launch_tz<StepParamsFF, 64>(e, q, nsteps);
            case 128: return ens_launch_tz<StepParamsFF, 128>(e, q, nsteps);
            default: return ens_launch_tz<StepParamsFF, 256>(e, q, nsteps);
        }
    }
    const StepParamsF q = f32_params(p);
    switch (e->tz) {
        case 64: return ens_launch_tz<StepParamsF, 64>(e, q, nsteps);
        case 128: return ens_launch_tz<StepParamsF, 128>(e, q, nsteps);
        default: return ens_launch_tz<StepParamsF, 256>(e, q, nsteps);
    }
}

static void ens_drop_graph(lbm_ensemble* e) {
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    e->gexec = nullptr;
    e->g_steps = 0;
}

extern "C" {

int lbm_ensemble_create(lbm_ensemble** out, int n, lbm_ctx* const* ctxs) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !ctxs) return fail(LBM_EINVAL, "need n >= 1 contexts");
    for (int i = 0; i < n; i++) {
        if (!ctxs[i]) return fail(LBM_EINVAL, "context %d is NULL", i);
        const lbm_ctx* a = ctxs[0];
        const lbm_ctx* b = ctxs[i];
        if (b->device != a->device || b->prec != a->prec || b->tau != a->tau || b->grav != a->grav ||
            b->stream != a->stream)
            return fail(LBM_EINVAL, "context %d differs from context 0 in device, precision, tau, g or stream", i);
        NEED_BOUNCE_BACK(b, "an ensemble");
    }
    NOT_DEV(ctxs[0], "an ensemble");
    if (ctxs[0]->prec != LBM_F64_FF && ctxs[0]->prec != LBM_F32)
        return fail(LBM_EINVAL, "ensembles take LBM_F64_FF or LBM_F32 contexts");
    DeviceGuard dg(ctxs[0]->device);
    lbm_ensemble* e = new lbm_ensemble();
    e->n = n;
    e->prec = ctxs[0]->prec;
    e->device = ctxs[0]->device;
    e->stream = ctxs[0]->stream;
    e->ctx.assign(ctxs, ctxs + n);
    bool ok = dev_malloc(&e->d_lats, n * sizeof(EnsLattice)) == cudaSuccess &&
              dev_malloc(&e->d_ctl, sizeof(EnsControl)) == cudaSuccess &&
              dev_malloc(&e->d_done, n * sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        cudaFree(e->d_lats); cudaFree(e->d_ctl); cudaFree(e->d_done);
        delete e;
        return fail(LBM_ENOMEM, "ensemble control allocation failed");
    }
    cudaMemset(e->d_ctl, 0, sizeof(EnsControl));
    *out = e;
    return LBM_OK;
}

int lbm_ensemble_destroy(lbm_ensemble* e) {
    if (!e) return LBM_OK;
    DeviceGuard dg(e->device);
    cudaStreamSynchronize(e->stream);
    ens_drop_graph(e);
    cudaFree(e->d_lats); cudaFree(e->d_ctl); cudaFree(e->d_done);
    delete e;
    return LBM_OK;
}

int lbm_ensemble_config(lbm_ensemble* e, int mode, int tile_z, int ctas_per_sm) {
    if (!e) return fail(LBM_EINVAL, "ensemble is NULL");
    if (mode != 0 && mode != 1) return fail(LBM_EINVAL, "mode must be 0 (per step) or 1 (persistent)");
    if (tile_z != 64 && tile_z != 128 && tile_z != 256) return fail(LBM_EINVAL, "tile_z must be 64, 128 or 256");
    if (ctas_per_sm < 0) return fail(LBM_EINVAL, "ctas_per_sm < 0");
    e->mode = mode;
    e->tz = tile_z;
    e->ctas_per_sm = ctas_per_sm;
    ens_drop_graph(e);
    return LBM_OK;
}

int lbm_ensemble_set_wait(lbm_ensemble* e, long long spin_limit_cycles, unsigned int extra_wait) {
    if (!e || spin_limit_cycles < 1) return fail(LBM_EINVAL, "bad arguments");
    e->spin_limit = spin_limit_cycles;
    e->extra_wait = extra_wait;
    ens_drop_graph(e);
    return LBM_OK;
}

int lbm_ensemble_step(lbm_ensemble* e, int nsteps) {
    if (!e) return fail(LBM_EINVAL, "ensemble is NULL");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    DeviceGuard dg(e->device);
    int rc = ens_layout(e);
    if (rc) return rc;
    rc = ens_launch(e, nsteps);
    if (rc) return rc;
    for (lbm_ctx* c : e->ctx) c->cur ^= (nsteps & 1);
    return LBM_OK;
}

int lbm_ensemble_sync(lbm_ensemble* e) {
    if (!e) return fail(LBM_EINVAL, "ensemble is NULL");
    DeviceGuard dg(e->device);
    CU(cudaStreamSynchronize(e->stream));
    EnsControl h;
    CU(cudaMemcpy(&h, e->d_ctl, sizeof h, cudaMemcpyDeviceToHost));
    if (h.err) {
        CU(cudaMemset(e->d_ctl, 0, sizeof h));
        return fail(LBM_ETIMEOUT, "persistent ensemble: a step barrier wait ran out (error word 0x%x)", h.err);
    }
    return LBM_OK;
}

int lbm_ensemble_capture(lbm_ensemble* e, int nsteps) {
    if (!e) return fail(LBM_EINVAL, "ensemble is NULL");
    if (nsteps < 1) return fail(LBM_EINVAL, "nsteps < 1");
    DeviceGuard dg(e->device);
    ens_drop_graph(e);
    int rc = ens_layout(e);
    if (rc) return rc;
    if (!e->stream) return fail(LBM_EINVAL, "graph capture needs a non-default stream");
    CU(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    rc = ens_launch(e, nsteps);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return fail(LBM_ECUDA, "stream capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&e->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        e->gexec = nullptr;
        return fail(LBM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    e->g_steps = nsteps;
    e->g_cur.clear();
    for (lbm_ctx* c : e->ctx) e->g_cur.push_back(c->cur);
    return LBM_OK;
}

int lbm_ensemble_graph_launch(lbm_ensemble* e) {
    if (!e || !e->gexec) return fail(LBM_ESTATE, "no captured graph");
    for (int i = 0; i < e->n; i++)
        if (e->ctx[i]->cur != e->g_cur[i])
            return fail(LBM_ESTATE, "lattice %d is not in the buffer the graph was captured for", i);
    DeviceGuard dg(e->device);
    CU(cudaGraphLaunch(e->gexec, e->stream));
    for (int i = 0; i < e->n; i++) e->ctx[i]->cur ^= (e->g_steps & 1);
    return LBM_OK;
}

int lbm_ensemble_tune(lbm_ensemble* e, int steps, double* best_ms, int* best_mode, int* best_tz, int* best_ctas) {
    if (!e || steps < 1) return fail(LBM_EINVAL, "bad arguments");
    DeviceGuard dg(e->device);
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    double best = 1e300;
    int bm = 1, bt = 128, bc = 0;
    const int tzs[3] = {64, 128, 256};
    for (int mode = 0; mode <= 1; mode++)
        for (int ti = 0; ti < 3; ti++)
            for (int ctas = (mode ? 1 : 0); ctas <= (mode ? 10 : 0); ctas++) {
                e->mode = mode; e->tz = tzs[ti]; e->ctas_per_sm = ctas;
                if (mode) {   // skip CTA counts beyond what fits
                    int per_sm = 0;
                    cudaError_t oe = (e->prec == LBM_F64_FF)
                        ? (tzs[ti] == 64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<StepParamsFF, 64>, 64, 0)
                           : tzs[ti] == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<StepParamsFF, 128>, 128, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<StepParamsFF, 256>, 256, 0))
                        : (tzs[ti] == 64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<StepParamsF, 64>, 64, 0)
                           : tzs[ti] == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<StepParamsF, 128>, 128, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<StepParamsF, 256>, 256, 0));
                    if (oe != cudaSuccess) return fail(LBM_ECUDA, "occupancy query failed");
                    if (ctas > per_sm) continue;
                }
                int rc = lbm_ensemble_step(e, steps);          // warm
                if (!rc) rc = lbm_ensemble_sync(e);
                if (rc) return rc;
                CU(cudaEventRecord(a, e->stream));
                rc = lbm_ensemble_step(e, steps);
                if (rc) return rc;
                CU(cudaEventRecord(b, e->stream));
                CU(cudaEventSynchronize(b));
                rc = lbm_ensemble_sync(e);
                if (rc) return rc;
                float ms = 0.f;
                CU(cudaEventElapsedTime(&ms, a, b));
                if (ms < best) { best = ms; bm = mode; bt = tzs[ti]; bc = ctas; }
            }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e->mode = bm; e->tz = bt; e->ctas_per_sm = bc;
    ens_drop_graph(e);
    if (best_ms) *best_ms = best / steps;
    if (best_mode) *best_mode = bm;
    if (best_tz) *best_tz = bt;
    if (best_ctas) *best_ctas = bc;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Allocation-free horizontal mean of T (lbm_row_mean_T_noalloc).
//
// For callers that must not allocate device memory: the two-stage reduction of
// lbm_row_mean_T keeps its per-chunk partial sums in this file-scope array instead of
// context scratch.  Host code cannot use the array's name as a device address; the
// address is taken once per device with cudaGetSymbolAddress, with that device current.
// ---------------------------------------------------------------------------------
#define LBM_NOALLOC_SCRATCH_DOUBLES (1 << 20)   /* 8 MiB per device, held until exit */

static __device__ __align__(256) double g_rowT_scratch[LBM_NOALLOC_SCRATCH_DOUBLES];

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[128];

// Per-device set-up: lattice constants and the scratch address (no allocation).
static int noalloc_setup(int dev, double** out) {
    if (dev < 0 || dev >= 128) return fail(LBM_EINVAL, "device index %d out of range", dev);
    int rc = upload_lattice(dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rowT_scratch);
        if (e != cudaSuccess || !p)
            return fail(LBM_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (double*)p;
    }
    *out = g_noalloc_ptr[dev];
    return LBM_OK;
}

extern "C" int lbm_row_mean_T_noalloc(const double* f, int Lx, int Lz, double* Tbar, void* cuda_stream) {
    if (!f || !Tbar) return fail(LBM_EINVAL, "NULL argument");
    if (Lx < 1 || Lz < 1) return fail(LBM_EINVAL, "lattice %d x %d: need Lx >= 1, Lz >= 1", Lx, Lz);
    if (Lz > LBM_NOALLOC_SCRATCH_DOUBLES)
        return fail(LBM_EINVAL, "Lz = %d exceeds the static scratch of %d rows", Lz, LBM_NOALLOC_SCRATCH_DOUBLES);
    if ((long long)Q * Lx * Lz >= (1LL << 31))
        return fail(LBM_EINVAL, "lattice %d x %d too large: 37*Lx*Lz must be < 2^31", Lx, Lz);
    int dev = -1;
    CU(cudaGetDevice(&dev));
    cudaPointerAttributes af, at;
    CU(cudaPointerGetAttributes(&af, f));
    CU(cudaPointerGetAttributes(&at, Tbar));
    if (af.type != cudaMemoryTypeDevice || at.type != cudaMemoryTypeDevice || af.device != dev || at.device != dev)
        return fail(LBM_EINVAL, "f and Tbar must be device memory on the current device %d", dev);
    double* scratch = nullptr;
    int rc = noalloc_setup(dev, &scratch);
    if (rc) return rc;
    // same chunking as lbm_row_mean_T, bounded by the static scratch
    const int target = std::max(1, std::min((148 * 16 * 128) / Lz, LBM_NOALLOC_SCRATCH_DOUBLES / Lz));
    const int nx_per = (Lx + std::min(Lx, target) - 1) / std::min(Lx, target);
    const int nch = (Lx + nx_per - 1) / nx_per;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    dim3 grid((Lz + 127) / 128, nch);
    k_rowT_partial<StoreF64><<<grid, 128, 0, st>>>(f, Lx, Lz, nx_per, scratch, LBM_NOALLOC_SCRATCH_DOUBLES);
    LAUNCH_CHECK();
    k_rowT_final<<<(Lz + 127) / 128, 128, 0, st>>>(scratch, LBM_NOALLOC_SCRATCH_DOUBLES, nch, Lx, Lz, Tbar);
    LAUNCH_CHECK();
    return LBM_OK;
}

// ---------------------------------------------------------------------------------
// x-slab decomposition of Sec. III.B (the paper's multi-GPU layout) on one device.
// Slab k owns the global columns [k Lxs, (k + 1) Lxs) and keeps them at local columns
// [HX, HX + Lxs) of a buffer of W = Lxs + 2 HX columns; local columns [0, HX) and
// [HX + Lxs, W) are halos holding the neighbours' edge columns (periodic in k), refreshed
// before every step, so the step kernels never wrap x inside a slab.
// Overlap mode (the paper's three-stream scheme): the bulk columns [2 HX, Lxs) need no
// halo and run on a second stream while the halo copies and then the edge columns
// [HX, 2 HX) and [Lxs, Lxs + HX) run on the context's stream.  Per step t (input B_t):
//   bulk stream: wait ev_comm[t-1]; bulk kernels;                   record ev_bulk[t]
//   comm stream: wait ev_bulk[t-1]; halo copies into B_t; edges;    record ev_comm[t]
// bulk(t) reads interior columns of B_t written by bulk(t-1) (same stream) and edge(t-1)
// (ev_comm), and writes B_{t+1} = B_{t-1}, which bulk(t-1) and edge(t-1) read; edge(t)
// reads B_t columns written by bulk(t-1) (ev_bulk) and writes B_{t-1}, read by bulk(t-1).
// ---------------------------------------------------------------------------------
namespace {
constexpr int HX = 3;   // halo columns = max |c_x|
}

struct lbm_slabs {
    lbm_ctx* c = nullptr;
    int n = 0, Lxs = 0, W = 0;
    size_t es = 0, slab_elems = 0;     // element size, Q * W * Lz elements per slab copy
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    cudaStream_t bulk = nullptr;
    cudaEvent_t ev_bulk[2] = {nullptr, nullptr}, ev_comm[2] = {nullptr, nullptr};
    long long t = 0;                   // steps taken (event parity)
};

static void slabs_free(lbm_slabs* s) {
    for (int i = 0; i < 2; i++) {
        if (s->buf[i]) cudaFree(s->buf[i]);
        if (s->ev_bulk[i]) cudaEventDestroy(s->ev_bulk[i]);
        if (s->ev_comm[i]) cudaEventDestroy(s->ev_comm[i]);
    }
    if (s->bulk) cudaStreamDestroy(s->bulk);
    delete s;
}

static char* slab_base(const lbm_slabs* s, int b, int k) {
    return (char*)s->buf[b] + (size_t)k * s->slab_elems * s->es;
}

// Halo columns of every slab of copy b from its neighbours' edge columns, on stream st.
static int slabs_exchange(lbm_slabs* s, int b, cudaStream_t st) {
    const size_t Lz = s->c->Lz;
    const size_t pitch = (size_t)s->W * Lz * s->es, width = (size_t)HX * Lz * s->es;
    for (int k = 0; k < s->n; k++) {
        const int km = (k + s->n - 1) % s->n, kp = (k + 1) % s->n;
        CU(cudaMemcpy2DAsync(slab_base(s, b, k), pitch, slab_base(s, b, km) + (size_t)s->Lxs * Lz * s->es, pitch,
                             width, Q, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpy2DAsync(slab_base(s, b, k) + (size_t)(HX + s->Lxs) * Lz * s->es, pitch,
                             slab_base(s, b, kp) + (size_t)HX * Lz * s->es, pitch, width, Q,
                             cudaMemcpyDeviceToDevice, st));
    }
    return LBM_OK;
}

// Interior columns between the context's current copy and the slabs' copy cur.
static int slabs_copy_interiors(lbm_slabs* s, bool to_slabs) {
    lbm_ctx* c = s->c;
    const size_t Lz = c->Lz;
    const size_t gpitch = (size_t)c->Lx * Lz * s->es, spitch = (size_t)s->W * Lz * s->es;
    const size_t width = (size_t)s->Lxs * Lz * s->es;
    for (int k = 0; k < s->n; k++) {
        char* g = (char*)c->buf[c->cur] + (size_t)k * s->Lxs * Lz * s->es;
        char* l = slab_base(s, s->cur, k) + (size_t)HX * Lz * s->es;
        if (to_slabs) CU(cudaMemcpy2DAsync(l, spitch, g, gpitch, width, Q, cudaMemcpyDeviceToDevice, c->stream));
        else CU(cudaMemcpy2DAsync(g, gpitch, l, spitch, width, Q, cudaMemcpyDeviceToDevice, c->stream));
    }
    return LBM_OK;
}

extern "C" {

int lbm_slabs_create(lbm_slabs** out, lbm_ctx* c, int nslab) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!c) return fail(LBM_EINVAL, "ctx is NULL");
    NEED_BOUNCE_BACK(c, "the slab decomposition");
    NOT_DEV(c, "the slab decomposition");
    if (nslab < 1 || c->Lx % nslab) return fail(LBM_EINVAL, "Lx = %d is not a multiple of nslab = %d", c->Lx, nslab);
    if (c->Lx / nslab < HX) return fail(LBM_EINVAL, "slabs of %d columns: need at least %d", c->Lx / nslab, HX);
    DeviceGuard dg(c->device);
    lbm_slabs* s = new lbm_slabs();
    s->c = c;
    s->n = nslab;
    s->Lxs = c->Lx / nslab;
    s->W = s->Lxs + 2 * HX;
    s->es = pop_bytes(c->prec);
    s->slab_elems = (size_t)Q * s->W * c->Lz;
    bool ok = (long long)s->slab_elems < (1LL << 31);
    for (int i = 0; ok && i < 2; i++)
        ok = dev_malloc(&s->buf[i], (size_t)nslab * s->slab_elems * s->es) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->ev_bulk[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->ev_comm[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->bulk, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        slabs_free(s);
        return fail(LBM_ENOMEM, "slab buffers or streams could not be created");
    }
    *out = s;
    return LBM_OK;
}

int lbm_slabs_destroy(lbm_slabs* s) {
    if (!s) return LBM_OK;
    DeviceGuard dg(s->c->device);
    cudaStreamSynchronize(s->c->stream);
    cudaStreamSynchronize(s->bulk);
    slabs_free(s);
    return LBM_OK;
}

int lbm_slabs_scatter(lbm_slabs* s) {
    if (!s) return fail(LBM_EINVAL, "slabs is NULL");
    DeviceGuard dg(s->c->device);
    int rc = slabs_copy_interiors(s, true);
    if (rc) return rc;
    s->t = 0;
    return LBM_OK;
}

int lbm_slabs_step(lbm_slabs* s, int nsteps, int overlap) {
    if (!s) return fail(LBM_EINVAL, "slabs is NULL");
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
    lbm_ctx* c = s->c;
    NEED_BOUNCE_BACK(c, "the slab decomposition");
    DeviceGuard dg(c->device);
    StepParams p = step_params(c);
    p.Lx = s->W;                      // the kernels address one slab buffer
    p.plane = s->W * c->Lz;
    const bool ov = overlap && s->Lxs > 2 * HX;
    const Tiling whole = make_tiling_cols(HX, s->Lxs, c->Lz, BLOCK_Z);
    const Tiling bulk = make_tiling_cols(2 * HX, s->Lxs - 2 * HX, c->Lz, BLOCK_Z);
    const Tiling edge_lo = make_tiling_cols(HX, HX, c->Lz, BLOCK_Z);
    const Tiling edge_hi = make_tiling_cols(s->Lxs, HX, c->Lz, BLOCK_Z);
    if (ov && s->t == 0) {            // first step: both streams start after the scatter
        CU(cudaEventRecord(s->ev_comm[1], c->stream));
        CU(cudaEventRecord(s->ev_bulk[1], c->stream));
    }
    for (int i = 0; i < nsteps; i++) {
        const int b = s->cur;
        if (!ov) {
            int rc = slabs_exchange(s, b, c->stream);
            if (rc) return rc;
            for (int k = 0; k < s->n; k++)
                launch_step(c->prec, slab_base(s, b, k), slab_base(s, b ^ 1, k), p, whole, c->stream);
            LAUNCH_CHECK();
        } else {
            const int now = (int)(s->t & 1), prev = now ^ 1;
            CU(cudaStreamWaitEvent(s->bulk, s->ev_comm[prev], 0));
            for (int k = 0; k < s->n; k++)
                launch_step(c->prec, slab_base(s, b, k), slab_base(s, b ^ 1, k), p, bulk, s->bulk);
            LAUNCH_CHECK();
            CU(cudaEventRecord(s->ev_bulk[now], s->bulk));
            CU(cudaStreamWaitEvent(c->stream, s->ev_bulk[prev], 0));
            int rc = slabs_exchange(s, b, c->stream);
            if (rc) return rc;
            for (int k = 0; k < s->n; k++) {
                launch_step(c->prec, slab_base(s, b, k), slab_base(s, b ^ 1, k), p, edge_lo, c->stream);
                launch_step(c->prec, slab_base(s, b, k), slab_base(s, b ^ 1, k), p, edge_hi, c->stream);
            }
            LAUNCH_CHECK();
            CU(cudaEventRecord(s->ev_comm[now], c->stream));
        }
        s->cur ^= 1;
        s->t++;
    }
    if (ov && nsteps > 0) CU(cudaStreamWaitEvent(c->stream, s->ev_bulk[(s->t - 1) & 1], 0));
    return LBM_OK;
}

int lbm_slabs_gather(lbm_slabs* s) {
    if (!s) return fail(LBM_EINVAL, "slabs is NULL");
    DeviceGuard dg(s->c->device);
    int rc = slabs_copy_interiors(s, false);
    if (rc) return rc;
    CU(cudaStreamSynchronize(s->c->stream));
    return LBM_OK;
}

}  // extern "C"
