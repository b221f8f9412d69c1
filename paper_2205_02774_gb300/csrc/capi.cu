// Host side of libstglbm.so: argument checks, the FP64 inlet setup
// (Algorithm 1, LBM section steps 1-4), device state, CUDA-graph step loop,
// readback and error reporting.  Declarations and conventions: stg_lbm.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "aa_layout.cuh"
#include "d3q19.cuh"
#include "handle.h"

using stg::StepCtl;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kCs = 0.57735026918962576451;  // sqrt(1/3)
thread_local std::string g_create_error;

}  // namespace

namespace stg {
// message for stg_lbm_last_error(NULL) from entry points without a handle
void record_error(const std::string &msg) { g_create_error = msg; }
}  // namespace stg

namespace stg {
namespace host {

int fail(stg_lbm *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(stg_lbm *h, cudaError_t e, const char *what)
{
    return fail(h, STG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace host
}  // namespace stg

using namespace stg::host;

namespace {

// Pinned host words for the mass read-backs, carved from blocks that are
// allocated once and kept: cudaMallocHost / cudaFreeHost per lattice could
// synchronise the device, which would stall the other lattices' work when
// jobs come and go.
struct PinnedSlots {
    std::mutex mu;
    std::vector<double *> free_slots;
    std::vector<void *> blocks;
    static constexpr int SLOT = 4, PER_BLOCK = 256;
    double *get()
    {
        std::lock_guard<std::mutex> lk(mu);
        if (free_slots.empty()) {
            void *b = nullptr;
            if (cudaMallocHost(&b, sizeof(double) * SLOT * PER_BLOCK) != cudaSuccess) return nullptr;
            blocks.push_back(b);
            for (int k = PER_BLOCK - 1; k >= 0; --k) free_slots.push_back(static_cast<double *>(b) + SLOT * k);
        }
        double *p = free_slots.back();
        free_slots.pop_back();
        return p;
    }
    void put(double *p)
    {
        std::lock_guard<std::mutex> lk(mu);
        free_slots.push_back(p);
    }
};
PinnedSlots &pinned_slots()
{
    static PinnedSlots *s = new PinnedSlots();  // kept for the process lifetime
    return *s;
}

#define CK(call)                                                \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);  \
    } while (0)

void *dalloc(stg_lbm *h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(bytes, h->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        h->allocs.emplace_back(p, bytes);
        h->info.device_bytes += (int64_t)bytes;
    }
    return p;
}

// SplitMix64 (Steele, Lea & Flood 2014): Weyl increment + 64-bit finaliser.
void splitmix_uniform(uint64_t seed, int32_t n, double *out)
{
    uint64_t state = seed;
    for (int32_t i = 0; i < n; ++i) {
        state += 0x9E3779B97F4A7C15ULL;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        out[i] = (double)(z >> 11) * 0x1.0p-53;
    }
}

// Piecewise-linear profile through (0, lo), the FV centres, (2h, hi).
struct Interp {
    const double *yc;
    int n;
    double top;
    double at(const double *v, int stride, int comp, double lo, double hi, double y) const
    {
        if (y <= yc[0]) return lo + (v[comp] - lo) * (y / yc[0]);
        if (y >= yc[n - 1]) {
            const double span = top - yc[n - 1];
            const double s = span > 0 ? (y - yc[n - 1]) / span : 0.0;
            return v[(size_t)(n - 1) * stride + comp] + (hi - v[(size_t)(n - 1) * stride + comp]) * s;
        }
        int lo_i = 0, hi_i = n - 1;  // bisection: yc[lo_i] <= y < yc[hi_i]
        while (hi_i - lo_i > 1) {
            const int mid = (lo_i + hi_i) / 2;
            if (yc[mid] <= y) lo_i = mid;
            else hi_i = mid;
        }
        const double s = (y - yc[lo_i]) / (yc[hi_i] - yc[lo_i]);
        const double a = v[(size_t)lo_i * stride + comp], b = v[(size_t)hi_i * stride + comp];
        return a + (b - a) * s;
    }
};

// A fraction of a turn, f in [0, 1), as a Q0.64 fixed-point number.
uint64_t turns_q64(double f)
{
    f -= std::floor(f);
    const double hi = std::floor(std::ldexp(f, 32));
    const double lo = std::floor(std::ldexp(std::ldexp(f, 32) - hi, 32));
    return ((uint64_t)hi << 32) | (uint64_t)lo;
}

// Modified von Karman spectrum of eq. (qn) (Shur et al.'s form, cited by the
// paper):
//   E(k) = (k/k_e)^4 [1 + 2.4 (k/k_e)^2]^(-17/6) exp(-(12 k/k_eta)^2)
//          exp(-(4 max(k - 0.9 k_cut, 0)/k_cut)^3),
// k_e = 2 pi/l_e, k_eta = 2 pi/l_eta, k_cut = 2 pi/l_cut; l_e <= 0 gives 0,
// l_eta <= 0 and l_cut <= 0 switch their factor off.
double vk_spectrum(double k, double le, double leta, double lcut)
{
    if (le <= 0.0) return 0.0;
    const double r = k * le / (2.0 * kPi);  // k / k_e
    const double r2 = r * r;
    double e = r2 * r2 * std::pow(1.0 + 2.4 * r2, -17.0 / 6.0);
    if (leta > 0.0) {
        const double g = 12.0 * k * leta / (2.0 * kPi);  // 12 k / k_eta
        e *= std::exp(-g * g);
    }
    if (lcut > 0.0) {
        const double kc = 2.0 * kPi / lcut;
        const double hh = 4.0 * std::max(k - 0.9 * kc, 0.0) / kc;
        e *= std::exp(-hh * hh * hh);
    }
    return e;
}

double wrap2pi(double v)
{
    v = std::fmod(v, 2.0 * kPi);
    return v < 0.0 ? v + 2.0 * kPi : v;
}

// Inlet tables: Algorithm 1, LBM section steps 1-4.
int build_inlet(stg_lbm *h, const stg_rans_profile *r, uint64_t seed)
{
    const int ny = h->d.ny, nz = h->d.nz;
    const stg_rans_profile &R = *r;
    // unit conversion, eqs. (c_factor), (u_transfer), (lbe-nu), (ma-eq)
    const double c_x = 2.0 * R.h_phys / ny;
    double Umax = 0.0;
    for (int i = 0; i < R.n_fv; ++i) Umax = std::max(Umax, R.U[i]);
    double c_t;
    if (R.mach_target > 0.0) {
        if (!(Umax > 0.0)) return fail(h, STG_ERR_INVALID, "mach_target needs max(U) > 0");
        c_t = R.mach_target * kCs * c_x / Umax;
    } else {
        c_t = (h->d.tau0 - 0.5) / 3.0 * c_x * c_x / R.nu_phys;
    }
    const double su = c_t / c_x;
    if (Umax * su / kCs >= 0.1)
        return fail(h, STG_ERR_INVALID, "lattice Mach number of the RANS maximum velocity is >= 0.1");
    h->info.c_x = c_x;
    h->info.c_t = c_t;
    h->info.U_b = R.U_bulk * su;

    Interp ip{R.y_c, R.n_fv, 2.0 * R.h_phys};
    std::vector<double> u_int(ny), R6(6 * (size_t)ny), le(ny), leta(ny), lcut(ny);
    double max_le = 0.0, max_kcut = 0.0;
    for (int j = 0; j < ny; ++j) {
        const double y = (j + 0.5) * c_x;
        const double U = ip.at(R.U, 1, 0, 0.0, 0.0, y);
        const double k = ip.at(R.k, 1, 0, 0.0, 0.0, y);
        const double eps = ip.at(R.eps, 1, 0, R.eps[0], R.eps[R.n_fv - 1], y);
        for (int c = 0; c < 6; ++c) R6[6 * (size_t)j + c] = ip.at(R.R, 6, c, 0.0, 0.0, y) * su * su;
        u_int[j] = U * su;
        // l_e = min(2 d_w, C_l l_t), l_t = k^{3/2}/eps; l_eta = (nu^3/eps)^{1/4}; lattice units
        const double dw = std::min(y, 2.0 * R.h_phys - y);
        const double lt = eps > 0.0 ? std::pow(std::max(k, 0.0), 1.5) / eps : 0.0;
        le[j] = std::min(2.0 * dw, h->p.C_l * lt) / c_x;
        leta[j] = eps > 0.0 ? std::pow(R.nu_phys * R.nu_phys * R.nu_phys / eps, 0.25) / c_x : 0.0;
        // eq. (lcut) with the lattice spacings (1, 1, 1)
        lcut[j] = 2.0 * std::min(std::max(1.0, 0.3) + 0.1 * dw / c_x, 1.0);
        max_le = std::max(max_le, le[j]);
        max_kcut = std::max(max_kcut, 2.0 * kPi / lcut[j]);
    }
    h->info.max_le = max_le;
    int N = 0;
    std::vector<double> kn, dk, phi, omg;
    std::vector<float> sig, A, B;
    if (max_le > 0.0) {
        const double kmin = kPi / max_le, kmax = 1.5 * max_kcut;
        h->info.k_min = kmin;
        h->info.k_max = kmax;
        N = h->p.n_modes > 0 ? h->p.n_modes
                             : (int)std::ceil(std::log(kmax / kmin) / std::log(1.0 + h->p.alpha) + 1.0);
        if (N < 1 || N > 100000) return fail(h, STG_ERR_INVALID, "mode count out of range");
        const double ratio = N > 1 ? std::pow(kmax / kmin, 1.0 / (N - 1)) : 1.0;
        kn.resize(N);
        dk.resize(N);
        for (int n = 0; n < N; ++n) {
            kn[n] = kmin * std::pow(ratio, (double)n);
            dk[n] = N > 1 ? kn[n] * (1.0 - 1.0 / ratio) : 1.0;
        }
        std::vector<double> u(4 * (size_t)N);
        splitmix_uniform(seed, 4 * N, u.data());
        sig.resize(3 * (size_t)N);
        phi.resize(N);
        omg.resize(N);
        A.resize((size_t)N * ny);
        B.resize((size_t)N * nz);
        for (int n = 0; n < N; ++n) {
            // eq. (dn): Phi, Theta = arccos(1 - 2 gamma), eta, phi
            const double Phi = 2.0 * kPi * u[4 * n + 0];
            const double Th = std::acos(1.0 - 2.0 * u[4 * n + 1]);
            const double eta = 2.0 * kPi * u[4 * n + 2];
            phi[n] = 2.0 * kPi * u[4 * n + 3];
            const double st = std::sin(Th), ct = std::cos(Th), sp = std::sin(Phi), cp = std::cos(Phi);
            const double se = std::sin(eta), ce = std::cos(eta);
            const double dx = st * cp, dy = st * sp, dz = ct;
            sig[3 * n + 0] = (float)(cp * ct * ce - sp * se);
            sig[3 * n + 1] = (float)(sp * ct * ce + cp * se);
            sig[3 * n + 2] = (float)(-st * ce);
            // eq. (psu) at x = 0: phase advance -2 pi d_x U_b / max l_e per step
            omg[n] = -2.0 * kPi * dx * h->info.U_b / max_le;
            for (int j = 0; j < ny; ++j) A[(size_t)n * ny + j] = (float)wrap2pi(kn[n] * dy * (j + 0.5));
            for (int k = 0; k < nz; ++k) B[(size_t)n * nz + k] = (float)wrap2pi(kn[n] * dz * k);
        }
    }
    h->N = N;
    h->info.n_modes = N;
    h->a_filter = h->p.T_filter > 0.0 ? (float)std::exp(-1.0 / h->p.T_filter) : 0.0f;
    h->info.a_filter = h->a_filter;

    // mode amplitudes sqrt(6 q^n(y_j)), eq. (qn), per inlet node, FP64 on the
    // host (terms added in mode order)
    std::vector<float> SQ((size_t)std::max(N, 1) * ny, 0.0f);
    {
        std::vector<double> e(std::max(N, 1));
        for (int j = 0; j < ny; ++j) {
            double total = 0.0;
            for (int n = 0; n < N; ++n) {
                e[n] = vk_spectrum(kn[n], le[j], leta[j], lcut[j]) * dk[n];
                total += e[n];
            }
            for (int n = 0; n < N; ++n) SQ[(size_t)n * ny + j] = total > 0.0 ? (float)std::sqrt(6.0 * e[n] / total) : 0.0f;
        }
    }
    // time part of the phase, phi^n + omega^n t, as Q0.64 fractions of a turn:
    // the device adds them in wrapping 64-bit integer arithmetic (exact modulo a
    // turn), so no floating point grows with the step count
    std::vector<unsigned long long> phq(std::max(N, 1), 0ull), omq(std::max(N, 1), 0ull);
    for (int n = 0; n < N; ++n) {
        phq[n] = turns_q64(phi[n] / (2.0 * kPi));
        omq[n] = turns_q64(omg[n] / (2.0 * kPi));
    }

    // device tables
    const size_t Nn = (size_t)std::max(N, 1);
    h->A = (float *)dalloc(h, sizeof(float) * Nn * ny);
    h->B = (float *)dalloc(h, sizeof(float) * Nn * nz);
    h->SQ = (float *)dalloc(h, sizeof(float) * Nn * ny);
    h->sig = (float *)dalloc(h, sizeof(float) * 3 * Nn);
    h->phq = (unsigned long long *)dalloc(h, sizeof(unsigned long long) * Nn);
    h->omq = (unsigned long long *)dalloc(h, sizeof(unsigned long long) * Nn);
    h->a6 = (float *)dalloc(h, sizeof(float) * 6 * ny);
    h->u_int = (float *)dalloc(h, sizeof(float) * ny);
    double *dR6 = (double *)dalloc(h, sizeof(double) * 6 * ny);
    if (!h->A || !h->B || !h->SQ || !h->sig || !h->phq || !h->omq || !h->a6 || !h->u_int || !dR6)
        return fail(h, STG_ERR_NOMEM, "device allocation of the inlet tables failed");
    std::vector<float> uf(ny);
    for (int j = 0; j < ny; ++j) uf[j] = (float)u_int[j];
    CK(cudaMemcpy(h->u_int, uf.data(), sizeof(float) * ny, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dR6, R6.data(), sizeof(double) * 6 * ny, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->SQ, SQ.data(), sizeof(float) * SQ.size(), cudaMemcpyHostToDevice));
    if (N > 0) {
        CK(cudaMemcpy(h->A, A.data(), sizeof(float) * A.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->B, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->sig, sig.data(), sizeof(float) * sig.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->phq, phq.data(), sizeof(unsigned long long) * N, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->omq, omq.data(), sizeof(unsigned long long) * N, cudaMemcpyHostToDevice));
    }
    // FP64 Cholesky of the Reynolds stress on the device (setup only)
    CK(stg::launch_setup_nodes(ny, dR6, h->a6, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return STG_OK;
}

// inlet plane of the step with this parity
float *ubc_plane(const stg_lbm *h, int parity)
{
    return h->ubc + (size_t)(parity & 1) * 3 * (size_t)h->d.ny * h->d.nz;
}

// where the populations of the current state live (for probes and block reads)
stg::LatticeView lattice_view(const stg_lbm *h)
{
    stg::LatticeView v{};
    v.nx = h->d.nx;
    v.ny = h->d.ny;
    v.nz = h->d.nz;
    v.bc_x = h->d.bc_x;
    v.bc_y = h->d.bc_y;
    v.aa = h->aa ? 1 : 0;
    v.P = h->P;
    v.t = h->t;
    return v;
}

stg::StepArgs step_args(const stg_lbm *h, int parity)
{
    stg::StepArgs a{};
    a.src = h->lat[parity];
    a.dst = h->lat[parity ^ 1];
    for (int i = 0; i < 19; ++i) {
        const char *sp = static_cast<const char *>(h->lat[parity]) + (size_t)i * h->P * h->elem;
        char *dp = static_cast<char *>(h->lat[parity ^ 1]) + (size_t)i * h->P * h->elem;
        const long long shift = (long long)(stg::cx_of(i) + stg::cy_of(i) * h->d.nx) * (long long)h->elem;
        a.srcp[i] = sp;
        a.srci[i] = sp - shift;
        a.srcy[i] = sp - (long long)stg::cy_of(i) * h->d.nx * (long long)h->elem;
        a.dstp[i] = dp;
    }
    a.nx = h->d.nx;
    a.ny = h->d.ny;
    a.nz = h->d.nz;
    a.P = (unsigned)h->P;
    a.bc_x = h->d.bc_x;
    a.bc_y = h->d.bc_y;
    a.tau0 = (float)h->d.tau0;
    a.kq = (float)(18.0 * std::sqrt(2.0) * h->d.c_smag);
    a.Fx = (float)h->d.force[0];
    a.Fy = (float)h->d.force[1];
    a.Fz = (float)h->d.force[2];
    a.has_force = (h->d.force[0] != 0.0 || h->d.force[1] != 0.0 || h->d.force[2] != 0.0);
    a.ubc = ubc_plane(h, parity);
    a.spf = h->spf;
    a.ctl = h->ctl;
    a.parity = parity;
    a.stats_every = h->d.stats_every;
    a.interior = h->interior;
    a.aa = h->aa ? 1 : 0;
    a.tile_layout = h->tile.interior_layout;
    a.tile_zc = h->tile.interior_zc;
    a.tile_wall_zc = h->tile.wall_zc;
    a.check_every = h->d.check_every;
    a.stat_mean = h->stat_mean;
    a.stat_rey = h->stat_rey;
    a.stat_part = h->stat_part;
    a.mass_partial = h->mass_partial;
    a.mass_counter = h->mass_counter;
    a.mass_out = h->mass_out;
    return a;
}

stg::InletArgs inlet_args(const stg_lbm *h, int parity)
{
    stg::InletArgs a{};
    a.ny = h->d.ny;
    a.nz = h->d.nz;
    a.N = h->N;
    a.A = h->A;
    a.B = h->B;
    a.SQ = h->SQ;
    a.sig = h->sig;
    a.phq = h->phq;
    a.omq = h->omq;
    a.a6 = h->a6;
    a.u_int = h->u_int;
    a.a_filter = h->a_filter;
    a.uf = h->uf;
    a.ubc = ubc_plane(h, parity ^ 1);  // the plane of the next step
    a.ahead = 1;
    a.ctl = h->ctl;
    a.parity = parity;
    return a;
}

}  // namespace

namespace stg {
namespace host {

bool is_stats_step(const stg_lbm *h, int64_t t)
{
    return h->d.stats_every > 0 && (t + 1) % h->d.stats_every == 0;
}

}  // namespace host
}  // namespace stg

namespace {

// one step with the given parity (the device reads the step index itself);
// `stats` selects the sampling-step kernel variant
}  // namespace

namespace stg {
namespace host {

cudaError_t enqueue_step(stg_lbm *h, int parity, bool stats)
{
    const stg::InletArgs in = inlet_args(h, parity);
    return stg::launch_step(step_args(h, parity), h->d.storage, h->d.collision, stats, h->stream, h->side,
                            h->ev_fork, h->ev_join,
                            h->inout ? &in : nullptr);
}

}  // namespace host
}  // namespace stg

namespace {

// Graph of `steps` steps starting with parity p0.  single_stats >= 0: one
// step with that sampling flag; otherwise step s samples when (s + 1) is a
// multiple of the sampling period (a block that starts at an aligned index).
int capture(stg_lbm *h, int p0, int steps, int single_stats, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < steps && e == cudaSuccess; ++s) {
        const bool st = single_stats >= 0 ? single_stats != 0
                                          : (h->d.stats_every > 0 && (s + 1) % h->d.stats_every == 0);
        e = enqueue_step(h, (p0 + s) & 1, st);
    }
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch during capture");
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    // upload now, so that the first replay costs no more than later ones
    e = cudaGraphUpload(*out, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphUpload");
    return STG_OK;
}

void destroy_graphs(stg_lbm *h)
{
    for (int p = 0; p < 2; ++p) {
        for (int q = 0; q < 2; ++q) {
            if (h->g_single[p][q]) cudaGraphExecDestroy(h->g_single[p][q]);
            h->g_single[p][q] = nullptr;
        }
        if (h->g_block[p]) cudaGraphExecDestroy(h->g_block[p]);
        h->g_block[p] = nullptr;
    }
}

// Single-step graphs by [parity][sampling] and the block graphs by parity.
int capture_all(stg_lbm *h)
{
    destroy_graphs(h);
    int rc = STG_OK;
    for (int p = 0; p < 2 && rc == STG_OK; ++p) {
        rc = capture(h, p, 1, 0, &h->g_single[p][0]);
        if (rc == STG_OK && h->d.stats_every > 0) rc = capture(h, p, 1, 1, &h->g_single[p][1]);
        if (rc == STG_OK && h->block_steps > 0) rc = capture(h, p, h->block_steps, -1, &h->g_block[p]);
    }
    return rc;
}

bool tile_ok(const stg_tile &t)
{
    return (t.interior_layout == 0 || t.interior_layout == 1) &&
           (t.interior_zc == 0 || t.interior_zc >= stg::MIN_ZC) && (t.wall_zc == 0 || t.wall_zc >= stg::MIN_ZC);
}

}  // namespace

namespace stg {
namespace host {

int wait_stream(stg_lbm *h)
{
    CK(cudaEventRecord(h->ev_done, h->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(h->ev_done);
        if (e == cudaSuccess) return STG_OK;
        if (e != cudaErrorNotReady) return cuda_fail(h, e, "cudaEventQuery");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > h->timeout_s) return fail(h, STG_ERR_TIMEOUT, "timed out waiting for the device");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
}

}  // namespace host
}  // namespace stg

namespace {

// Evaluate the last completed mass check (non-blocking).
}  // namespace

namespace stg {
namespace host {

int poll_check(stg_lbm *h)
{
    if (!h->check_pending) return STG_OK;
    cudaError_t e = cudaEventQuery(h->ev_check);
    if (e == cudaErrorNotReady) return STG_OK;
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventQuery");
    h->check_pending = false;
    const double m = h->h_pinned[0];
    if (!std::isfinite(m)) {
        h->sticky = STG_ERR_UNSTABLE;
        return fail(h, STG_ERR_UNSTABLE, "non-finite mass at the last check");
    }
    if (h->d.mass_tol > 0.0 && std::fabs(m / h->mass0 - 1.0) > h->d.mass_tol) {
        h->sticky = STG_ERR_UNSTABLE;
        char buf[160];
        std::snprintf(buf, sizeof buf, "mass drift %.3e exceeds %.3e", m / h->mass0 - 1.0, h->d.mass_tol);
        return fail(h, STG_ERR_UNSTABLE, buf);
    }
    return STG_OK;
}

}  // namespace host
}  // namespace stg

namespace {

}  // namespace

namespace stg {
namespace host {

int queue_check_readback(stg_lbm *h, int64_t t_before)
{
    (void)t_before;
    // read back the last check only once a check step has run since the reset
    if (h->d.check_every > 0 && h->t / h->d.check_every > h->t0_stats / h->d.check_every) {
        CK(cudaMemcpyAsync(h->h_pinned, h->mass_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaEventRecord(h->ev_check, h->stream));
        h->check_pending = true;
    }
    return STG_OK;
}

}  // namespace host
}  // namespace stg

namespace {

// Rows of an in-place lattice after t completed steps to or from the
// canonical arrangement (f*_i(x) in slot i of cell x; aa_layout.cuh): plane
// swap for even t, shifted rows for odd t.  T is the element type (4 or 2
// bytes, copied bit for bit).
template <typename T>
void aa_convert(const stg_lbm *h, int64_t t, const T *src, T *dst, bool to_canonical)
{
    const int nx = h->d.nx, ny = h->d.ny, nz = h->d.nz;
    const size_t P = h->P;
    const bool px = h->d.bc_x == STG_BC_X_PERIODIC, py = h->d.bc_y == STG_BC_Y_PERIODIC;
    for (int i = 0; i < 19; ++i) {
        const int o = stg::opp_of(i), cx = stg::cx_of(i), cy = stg::cy_of(i), cz = stg::cz_of(i);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y) {
                const size_t row = ((size_t)z * ny + y) * nx;
                // canonical row (i, y, z) and the stored slots its elements map to
                auto canon = [&](int x) -> size_t { return (size_t)i * P + row + x; };
                auto own = [&](int x) -> size_t { return (size_t)o * P + row + x; };
                auto move = [&](size_t c, size_t s) {
                    if (to_canonical) dst[c] = src[s];
                    else dst[s] = src[c];
                };
                if ((t & 1) == 0) {
                    for (int x = 0; x < nx; ++x) move(canon(x), own(x));
                    continue;
                }
                int yt = y + cy, zt = z + cz;
                zt = zt < 0 ? zt + nz : (zt >= nz ? zt - nz : zt);
                if (py) yt = yt < 0 ? yt + ny : (yt >= ny ? yt - ny : yt);
                if (yt < 0 || yt >= ny) {
                    for (int x = 0; x < nx; ++x) move(canon(x), own(x));
                    continue;
                }
                const size_t trow = (size_t)i * P + ((size_t)zt * ny + yt) * nx;
                for (int x = 0; x < nx; ++x) {
                    int xt = x + cx;
                    if (px) xt = xt < 0 ? xt + nx : (xt >= nx ? xt - nx : xt);
                    if (xt < 0 || xt >= nx) move(canon(x), own(x));
                    else move(canon(x), trow + xt);
                }
            }
    }
}

int compute_mass(stg_lbm *h, double *out)
{
    stg::MassArgs m{};
    m.src = h->lat[h->t & 1];
    m.P = (unsigned)h->P;
    m.storage = h->d.storage;
    m.partial = h->m_partial;
    m.counter = h->m_counter;
    m.out = h->m_out;
    CK(stg::launch_mass(m, h->stream));
    CK(cudaMemcpyAsync(h->h_pinned + 1, h->m_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int rc = wait_stream(h);
    if (rc) return rc;
    *out = h->h_pinned[1];
    return STG_OK;
}

int reset_counters(stg_lbm *h, int64_t step)
{
    StepCtl c{};
    c.t[step & 1] = step;
    c.t[(step + 1) & 1] = step;
    c.t0_filter = step;
    CK(cudaMemcpyAsync(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice, h->stream));
    const size_t m = (size_t)h->d.nx * h->d.ny;
    CK(cudaMemsetAsync(h->stat_mean, 0, sizeof(double) * 3 * m, h->stream));
    CK(cudaMemsetAsync(h->stat_rey, 0, sizeof(double) * 6 * m, h->stream));
    CK(cudaMemsetAsync(h->mass_out, 0, sizeof(double) * 2, h->stream));
    if (h->inout) {
        // the inlet plane of the restart step (later planes are computed one step ahead)
        stg::InletArgs in = inlet_args(h, (int)(step & 1));
        in.ubc = ubc_plane(h, (int)(step & 1));
        in.ahead = 0;
        CK(stg::launch_inlet(in, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    h->t = step;
    h->t0_stats = step;
    h->check_pending = false;
    h->sticky = STG_OK;
    return STG_OK;
}

void release(stg_lbm *h)
{
    if (!h) return;
    if (h->batch) batch_detach(h);
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    for (auto &a : h->allocs) {
        if (h->has_alloc) h->alloc.free(a.first, a.second, h->alloc.ctx);
        else cudaFree(a.first);
    }
    h->allocs.clear();
    if (h->h_pinned) pinned_slots().put(h->h_pinned);
    if (h->ev_check) cudaEventDestroy(h->ev_check);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int validate(const stg_domain *d, const stg_rans_profile *r, const stg_params *p)
{
    if (!d) return fail(nullptr, STG_ERR_INVALID, "domain is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(nullptr, STG_ERR_INVALID, "lattice sizes must be >= 1");
    const double cells = (double)d->nx * d->ny * d->nz;
    if (cells > 2147483647.0) return fail(nullptr, STG_ERR_INVALID, "more than 2^31-1 cells");
    if (d->ny > 65535) return fail(nullptr, STG_ERR_INVALID, "ny must be <= 65535");
    if (d->storage != STG_FP32 && d->storage != STG_FP16_SHIFTED && d->storage != STG_FP16_SHIFTED_SR)
        return fail(nullptr, STG_ERR_INVALID, "bad storage");
    if (d->collision != STG_REGULARIZED && d->collision != STG_BGK) return fail(nullptr, STG_ERR_INVALID, "bad collision");
    if (d->bc_x != STG_BC_X_INLET_OUTLET && d->bc_x != STG_BC_X_PERIODIC) return fail(nullptr, STG_ERR_INVALID, "bad bc_x");
    if (d->bc_y != STG_BC_Y_WALLS && d->bc_y != STG_BC_Y_PERIODIC) return fail(nullptr, STG_ERR_INVALID, "bad bc_y");
    if (!(d->tau0 > 0.5) || !std::isfinite(d->tau0)) return fail(nullptr, STG_ERR_INVALID, "tau0 must be > 1/2");
    if (!(d->c_smag >= 0.0) || !std::isfinite(d->c_smag)) return fail(nullptr, STG_ERR_INVALID, "c_smag must be >= 0");
    if (d->stats_every < 0 || d->check_every < 0) return fail(nullptr, STG_ERR_INVALID, "negative cadence");
    if (d->streaming != STG_STREAM_PULL && d->streaming != STG_STREAM_AA) return fail(nullptr, STG_ERR_INVALID, "bad streaming");
    if (d->streaming == STG_STREAM_AA && (d->nx % 2 != 0 || d->nx < 4 || 19.0 * cells >= 4294967296.0))
        return fail(nullptr, STG_ERR_INVALID, "in-place streaming needs an even nx >= 4 and 19 nx ny nz < 2^32");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->force[a])) return fail(nullptr, STG_ERR_INVALID, "non-finite force");
    if (!(d->sponge_len >= 0.0) || !std::isfinite(d->sponge_len))
        return fail(nullptr, STG_ERR_INVALID, "sponge_len must be finite and >= 0");
    if (d->sponge_len > 0.0) {
        if (!(d->sponge_K >= 0.0) || !std::isfinite(d->sponge_K) || !(d->sponge_p >= 0.0) || !std::isfinite(d->sponge_p))
            return fail(nullptr, STG_ERR_INVALID, "sponge K and p must be finite and >= 0");
        if (d->force[0] != 0.0 || d->force[1] != 0.0 || d->force[2] != 0.0)
            return fail(nullptr, STG_ERR_INVALID, "a sponge zone needs force = 0");
    }
    if (d->bc_x == STG_BC_X_INLET_OUTLET) {
        if (d->nx < 3) return fail(nullptr, STG_ERR_INVALID, "inlet/outlet needs nx >= 3");
        if (!r || !p) return fail(nullptr, STG_ERR_INVALID, "inlet/outlet needs a RANS profile and STG parameters");
        if (r->n_fv < 2 || !r->y_c || !r->U || !r->k || !r->eps || !r->R)
            return fail(nullptr, STG_ERR_INVALID, "RANS profile needs n_fv >= 2 and all arrays");
        if (!(r->h_phys > 0.0) || !(r->nu_phys > 0.0) || !(r->mach_target >= 0.0) || !std::isfinite(r->U_bulk))
            return fail(nullptr, STG_ERR_INVALID, "RANS scalars out of range");
        for (int i = 0; i < r->n_fv; ++i) {
            if (!(r->y_c[i] > 0.0 && r->y_c[i] < 2.0 * r->h_phys) || (i > 0 && !(r->y_c[i] > r->y_c[i - 1])))
                return fail(nullptr, STG_ERR_INVALID, "y_c must increase strictly inside (0, 2 h_phys)");
            if (!std::isfinite(r->U[i]) || !(r->k[i] >= 0.0) || !(r->eps[i] >= 0.0))
                return fail(nullptr, STG_ERR_INVALID, "RANS U, k, eps must be finite, k and eps >= 0");
            for (int c = 0; c < 6; ++c)
                if (!std::isfinite(r->R[6 * (size_t)i + c])) return fail(nullptr, STG_ERR_INVALID, "non-finite R");
        }
        if (!(p->C_l > 0.0) || !(p->alpha > 0.0) || !(p->T_filter >= 0.0) || p->n_modes < 0)
            return fail(nullptr, STG_ERR_INVALID, "STG parameters out of range");
    }
    return STG_OK;
}

}  // namespace

extern "C" {

int stg_lbm_create(const stg_domain *domain, const stg_rans_profile *rans, const stg_params *stgp, uint64_t seed,
                   const stg_allocator *alloc, void *stream, stg_lbm **out)
{
    const Range range("stg_lbm_create");
    if (!out) return fail(nullptr, STG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int rc = validate(domain, rans, stgp);
    if (rc) return rc;
    stg_lbm *h = new stg_lbm();
    h->d = *domain;
    if (stgp) h->p = *stgp;
    h->inout = domain->bc_x == STG_BC_X_INLET_OUTLET;
    if (alloc && alloc->alloc && alloc->free) {
        h->alloc = *alloc;
        h->has_alloc = true;
    }
    auto bail = [&](int code) {
        g_create_error = h->err;
        release(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        h->err = "no CUDA device";
        return bail(STG_ERR_CUDA);
    }
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            h->err = "cudaStreamCreate failed";
            return bail(STG_ERR_CUDA);
        }
        h->own_stream = true;
    }
    int lo_prio = 0, hi_prio = 0;  // the branch (wall rows, inlet plane) gets the highest priority: its blocks start first
    if (cudaEventCreateWithFlags(&h->ev_check, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        !(h->h_pinned = pinned_slots().get())) {
        h->err = "event / pinned allocation failed";
        return bail(STG_ERR_CUDA);
    }
    const int nx = domain->nx, ny = domain->ny, nz = domain->nz;
    if (const char *ev = std::getenv("STG_LBM_INTERIOR")) {
        const std::string v(ev);
        h->interior = v == "scalar" ? 1 : v == "pair" ? 2 : 0;
    }
    h->P = (size_t)nx * ny * nz;
    h->elem = domain->storage == STG_FP32 ? 4 : 2;
    h->aa = domain->streaming == STG_STREAM_AA;
    h->lat[0] = dalloc(h, 19 * h->P * h->elem);
    h->lat[1] = h->aa ? h->lat[0] : dalloc(h, 19 * h->P * h->elem);  // in place: one lattice
    h->ubc = (float *)dalloc(h, sizeof(float) * 6 * (size_t)ny * nz);
    h->uf = (float *)dalloc(h, sizeof(float) * 3 * (size_t)ny * nz);
    h->ctl = (StepCtl *)dalloc(h, sizeof(StepCtl));
    h->stat_mean = (double *)dalloc(h, sizeof(double) * 3 * (size_t)nx * ny);
    h->stat_rey = (double *)dalloc(h, sizeof(double) * 6 * (size_t)nx * ny);
    h->mass_partial = (double *)dalloc(h, sizeof(double) * stg::step_grid_blocks(nx, ny, nz));
    if (domain->stats_every > 0) {
        h->stat_part = (float *)dalloc(h, sizeof(float) * 9 * (size_t)nx * ny * ((nz + stg::STAT_GROUP - 1) / stg::STAT_GROUP));
        if (!h->stat_part) {
            h->err = "device allocation failed";
            return bail(STG_ERR_NOMEM);
        }
    }
    h->mass_counter = (unsigned *)dalloc(h, sizeof(unsigned) * 4);
    h->mass_out = (double *)dalloc(h, sizeof(double) * 2);
    h->m_partial = (double *)dalloc(h, sizeof(double) * stg::mass_grid_blocks());
    h->m_counter = (unsigned *)dalloc(h, sizeof(unsigned) * 4);
    h->m_out = (double *)dalloc(h, sizeof(double) * 2);
    if (domain->sponge_len > 0.0) {
        // eq. (sponge_visco): factor per column, FP64 on the host
        std::vector<float> f(nx);
        const double xe = nx - 1.0, xs = xe - domain->sponge_len;
        for (int x = 0; x < nx; ++x) {
            const double xi = (x - xs) / (xe - xs);
            f[x] = x < xs ? 1.0f : (float)(domain->sponge_K * std::pow(xi, domain->sponge_p) + 1.0);
        }
        h->spf = (float *)dalloc(h, sizeof(float) * nx);
        if (!h->spf || cudaMemcpy(h->spf, f.data(), sizeof(float) * nx, cudaMemcpyHostToDevice) != cudaSuccess) {
            h->err = "sponge table";
            return bail(STG_ERR_NOMEM);
        }
    }
    if (!h->lat[0] || !h->lat[1] || !h->ubc || !h->uf || !h->ctl || !h->stat_mean || !h->stat_rey ||
        !h->mass_partial || !h->mass_counter || !h->mass_out || !h->m_partial || !h->m_counter || !h->m_out) {
        h->err = "device allocation failed";
        return bail(STG_ERR_NOMEM);
    }
    cudaError_t e = cudaSuccess;
    e = cudaMemsetAsync(h->mass_counter, 0, sizeof(unsigned) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->m_counter, 0, sizeof(unsigned) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->mass_out, 0, sizeof(double) * 2, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ubc, 0, sizeof(float) * 6 * (size_t)ny * nz, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->uf, 0, sizeof(float) * 3 * (size_t)ny * nz, h->stream);
    if (e != cudaSuccess) {
        cuda_fail(h, e, "cudaMemsetAsync");
        return bail(STG_ERR_CUDA);
    }
    if (h->inout) {
        rc = build_inlet(h, rans, seed);
        if (rc) return bail(rc);
    }
    // in place, the state before a step of even index keeps f*_i in slot opp(i)
    e = stg::launch_init_equilibrium(h->lat[0], domain->storage, nx, ny, nz, h->inout ? h->u_int : nullptr,
                                     h->aa ? 1 : 0, h->stream);
    if (e != cudaSuccess) {
        cuda_fail(h, e, "init kernel");
        return bail(STG_ERR_CUDA);
    }
    rc = reset_counters(h, 0);
    if (rc) return bail(rc);
    rc = compute_mass(h, &h->mass0);
    if (rc) return bail(rc);
    // block length: a multiple of the sampling period, at least 16 steps
    const int k = domain->stats_every;
    h->block_steps = k > 0 ? k * ((16 + k - 1) / k) : 16;
    if (h->block_steps > 256) h->block_steps = 0;  // very long sampling periods: single-step graphs only
    rc = capture_all(h);
    if (rc) return bail(rc);
    *out = h;
    return STG_OK;
}

int stg_lbm_estimate_bytes(const stg_domain *d, const stg_params *p, int64_t *bytes)
{
    if (!d || !bytes || d->nx < 1 || d->ny < 1 || d->nz < 1 ||
        (d->storage != STG_FP32 && d->storage != STG_FP16_SHIFTED && d->storage != STG_FP16_SHIFTED_SR))
        return fail(nullptr, STG_ERR_INVALID, "estimate: bad domain");
    auto r = [](double b) { return (double)(((int64_t)std::max(b, 16.0) + 255) & ~int64_t(255)); };
    const double nx = d->nx, ny = d->ny, nz = d->nz, P = nx * ny * nz;
    const double elem = d->storage == STG_FP32 ? 4.0 : 2.0;
    const double lattices = d->streaming == STG_STREAM_AA ? 1.0 : 2.0;
    double b = lattices * r(19 * P * elem) + r(24 * ny * nz) + r(12 * ny * nz) + r(sizeof(StepCtl)) + r(24 * nx * ny) + r(48 * nx * ny) +
               r(8.0 * stg::step_grid_blocks(d->nx, d->ny, d->nz)) + 2 * r(16) + 2 * r(16) +
               r(8.0 * stg::mass_grid_blocks());
    if (d->sponge_len > 0.0) b += r(4 * nx);
    if (d->stats_every > 0) b += r(36.0 * nx * ny * std::ceil(nz / (double)stg::STAT_GROUP));
    if (d->bc_x == STG_BC_X_INLET_OUTLET) {
        double N = 1.0;
        if (p && p->n_modes > 0) N = p->n_modes;
        else if (p && p->alpha > 0.0) N = std::ceil(std::log(1.5 * std::max(ny, 2.0)) / std::log(1.0 + p->alpha) + 1.0);
        // A, B, SQ, sigma, the two phase words, a6, u_int, the FP64 stresses
        b += r(4 * N * ny) + r(4 * N * nz) + r(4 * N * ny) + r(12 * N) + 2 * r(8 * N) + r(24 * ny) + r(4 * ny) +
             r(48 * ny);
    }
    *bytes = (int64_t)b;
    return STG_OK;
}

int stg_lbm_step(stg_lbm *h, int64_t n)
{
    const Range range("stg_lbm_step");
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; step the batch");
    if (n < 0) return fail(h, STG_ERR_INVALID, "negative step count");
    int rc = poll_check(h);
    if (rc) return rc;
    if (h->sticky) return fail(h, h->sticky, "an earlier check failed; reset the state first");
    const int per = h->d.stats_every;
    while (n > 0) {
        cudaGraphExec_t g;
        int k = 1;
        const int par = (int)(h->t & 1);
        const bool aligned = per <= 0 || h->t % per == 0;
        if (h->block_steps > 0 && n >= h->block_steps && aligned) {
            g = h->g_block[par];
            k = h->block_steps;
        } else {
            g = h->g_single[par][is_stats_step(h, h->t) ? 1 : 0];
        }
        CK(cudaGraphLaunch(g, h->stream));
        h->t += k;
        n -= k;
    }
    return queue_check_readback(h, h->t);
}

int stg_lbm_step_timed(stg_lbm *h, int64_t n, double *ms_step, double *ms_inlet)
{
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; step the batch");
    if (n < 1 || n > 4096) return fail(h, STG_ERR_INVALID, "step_timed needs 1 <= n <= 4096");
    if (h->sticky) return fail(h, h->sticky, "an earlier check failed; reset the state first");
    std::vector<cudaEvent_t> ev(3 * (size_t)n, nullptr);
    int rc = STG_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) rc = fail(h, STG_ERR_CUDA, "cudaEventCreate");
    for (int64_t s = 0; s < n && rc == STG_OK; ++s) {
        const int parity = (int)(h->t & 1);
        cudaError_t e = cudaEventRecord(ev[3 * s], h->stream);
        if (e == cudaSuccess && h->inout) e = stg::launch_inlet(inlet_args(h, parity), h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + 1], h->stream);
        if (e == cudaSuccess)
            e = stg::launch_step(step_args(h, parity), h->d.storage, h->d.collision, is_stats_step(h, h->t),
                                 h->stream, h->side, h->ev_fork, h->ev_join);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + 2], h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "timed step launch");
        else h->t += 1;
    }
    if (rc == STG_OK) rc = wait_stream(h);
    double sum_s = 0.0, sum_i = 0.0;
    if (rc == STG_OK) {
        for (int64_t s = 0; s < n; ++s) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
            cudaEventElapsedTime(&b, ev[3 * s + 1], ev[3 * s + 2]);
            sum_i += a;
            sum_s += b;
        }
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (rc) return rc;
    if (ms_step) *ms_step = sum_s / (double)n;
    if (ms_inlet) *ms_inlet = sum_i / (double)n;
    return STG_OK;
}

int stg_lbm_stats(stg_lbm *h, stg_stats *out)
{
    const Range range("stg_lbm_stats");
    if (!h || !out) return fail(h, STG_ERR_INVALID, "NULL argument");
    int rc = wait_stream(h);
    if (rc) return rc;
    rc = poll_check(h);
    const size_t m = (size_t)h->d.nx * h->d.ny;
    if (out->mean_sum) CK(cudaMemcpy(out->mean_sum, h->stat_mean, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost));
    if (out->rey_sum) CK(cudaMemcpy(out->rey_sum, h->stat_rey, sizeof(double) * 6 * m, cudaMemcpyDeviceToHost));
    out->step = h->t;
    const int64_t k = h->d.stats_every;
    out->n_samples = k > 0 ? (h->t / k - h->t0_stats / k) : 0;
    out->mass0 = h->mass0;
    unsigned long long kerr = 0;
    CK(cudaMemcpy(&kerr, &h->ctl->err, sizeof kerr, cudaMemcpyDeviceToHost));
    if (kerr) {
        h->sticky = STG_ERR_TIMEOUT;
        return fail(h, STG_ERR_TIMEOUT, "a kernel set its error bit (a bounded device-side wait expired)");
    }
    double mass = 0.0;
    int rc2 = compute_mass(h, &mass);
    if (rc2) return rc2;
    out->mass = mass;
    if (rc) return rc;
    if (!std::isfinite(mass)) {
        h->sticky = STG_ERR_UNSTABLE;
        return fail(h, STG_ERR_UNSTABLE, "non-finite mass");
    }
    return h->sticky;
}

int stg_lbm_reset_stats(stg_lbm *h)
{
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; remove it first");
    int rc = wait_stream(h);
    if (rc) return rc;
    const size_t m = (size_t)h->d.nx * h->d.ny;
    CK(cudaMemsetAsync(h->stat_mean, 0, sizeof(double) * 3 * m, h->stream));
    CK(cudaMemsetAsync(h->stat_rey, 0, sizeof(double) * 6 * m, h->stream));
    h->t0_stats = h->t;
    return wait_stream(h);
}

int stg_lbm_get_state(stg_lbm *h, void *host, size_t bytes)
{
    if (!h || !host) return fail(h, STG_ERR_INVALID, "NULL argument");
    if (bytes != 19 * h->P * h->elem) return fail(h, STG_ERR_INVALID, "state size mismatch");
    int rc = wait_stream(h);
    if (rc) return rc;
    if (!h->aa) {
        CK(cudaMemcpy(host, h->lat[h->t & 1], bytes, cudaMemcpyDeviceToHost));
        return STG_OK;
    }
    // in place: the stored arrangement depends on the step parity
    std::vector<unsigned char> raw(bytes);
    CK(cudaMemcpy(raw.data(), h->lat[0], bytes, cudaMemcpyDeviceToHost));
    if (h->elem == 4)
        aa_convert(h, h->t, reinterpret_cast<const uint32_t *>(raw.data()), static_cast<uint32_t *>(host), true);
    else
        aa_convert(h, h->t, reinterpret_cast<const uint16_t *>(raw.data()), static_cast<uint16_t *>(host), true);
    return STG_OK;
}

int stg_lbm_set_state(stg_lbm *h, const void *host, size_t bytes, int64_t step)
{
    if (!h || !host) return fail(h, STG_ERR_INVALID, "NULL argument");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; remove it first");
    if (bytes != 19 * h->P * h->elem) return fail(h, STG_ERR_INVALID, "state size mismatch");
    if (step < 0) return fail(h, STG_ERR_INVALID, "negative step");
    int rc = wait_stream(h);
    if (rc) return rc;
    if (!h->aa) {
        CK(cudaMemcpy(h->lat[step & 1], host, bytes, cudaMemcpyHostToDevice));
    } else {
        std::vector<unsigned char> raw(bytes);
        if (h->elem == 4)
            aa_convert(h, step, static_cast<const uint32_t *>(host), reinterpret_cast<uint32_t *>(raw.data()), false);
        else
            aa_convert(h, step, static_cast<const uint16_t *>(host), reinterpret_cast<uint16_t *>(raw.data()), false);
        CK(cudaMemcpy(h->lat[0], raw.data(), bytes, cudaMemcpyHostToDevice));
    }
    rc = reset_counters(h, step);
    if (rc) return rc;
    return compute_mass(h, &h->mass0);
}

}  // extern "C"

namespace {

// Checkpoint image: header, current populations, inlet filter state, FP64
// statistics sums.
struct CkptHeader {
    char magic[8];
    int32_t nx, ny, nz, storage;
    int64_t t, t0_stats, t0_filter;
    double mass0;
    int64_t pop_bytes, uf_bytes, stat_bytes, plane_bytes;
    int64_t streaming;  // stg_domain.streaming of the lattice (0 in images without it)
    int64_t reserved[4];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header layout");
constexpr char kCkptMagic[8] = {'S', 'T', 'G', 'C', 'K', 'P', 'T', '2'};

size_t ckpt_bytes(const stg_lbm *h)
{
    return sizeof(CkptHeader) + 19 * h->P * h->elem + sizeof(float) * 6 * (size_t)h->d.ny * h->d.nz +
           sizeof(double) * 9 * (size_t)h->d.nx * h->d.ny;
}

}  // namespace

extern "C" {

int stg_lbm_checkpoint_bytes(const stg_lbm *h, size_t *bytes)
{
    if (!h || !bytes) return STG_ERR_INVALID;
    *bytes = ckpt_bytes(h);
    return STG_OK;
}

int stg_lbm_save(stg_lbm *h, void *host, size_t bytes)
{
    const Range range("stg_lbm_save");
    if (!h || !host) return fail(h, STG_ERR_INVALID, "NULL argument");
    if (bytes != ckpt_bytes(h)) return fail(h, STG_ERR_INVALID, "checkpoint size mismatch");
    int rc = wait_stream(h);
    if (rc) return rc;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.nx = h->d.nx;
    hd.ny = h->d.ny;
    hd.nz = h->d.nz;
    hd.storage = h->d.storage;
    hd.t = h->t;
    hd.t0_stats = h->t0_stats;
    StepCtl c{};
    CK(cudaMemcpy(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost));
    hd.t0_filter = c.t0_filter;
    hd.mass0 = h->mass0;
    hd.pop_bytes = (int64_t)(19 * h->P * h->elem);
    hd.uf_bytes = (int64_t)(sizeof(float) * 3 * (size_t)h->d.ny * h->d.nz);
    hd.stat_bytes = (int64_t)(sizeof(double) * 9 * (size_t)h->d.nx * h->d.ny);
    hd.plane_bytes = hd.uf_bytes;
    hd.streaming = h->d.streaming;  // the populations are stored in the lattice's own arrangement
    char *p = static_cast<char *>(host);
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    CK(cudaMemcpy(p, h->lat[h->t & 1], hd.pop_bytes, cudaMemcpyDeviceToHost));
    p += hd.pop_bytes;
    CK(cudaMemcpy(p, h->uf, hd.uf_bytes, cudaMemcpyDeviceToHost));
    p += hd.uf_bytes;
    CK(cudaMemcpy(p, ubc_plane(h, (int)(h->t & 1)), hd.plane_bytes, cudaMemcpyDeviceToHost));  // this step's inlet plane
    p += hd.plane_bytes;
    const size_t m = (size_t)h->d.nx * h->d.ny;
    CK(cudaMemcpy(p, h->stat_mean, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(p + sizeof(double) * 3 * m, h->stat_rey, sizeof(double) * 6 * m, cudaMemcpyDeviceToHost));
    return STG_OK;
}

int stg_lbm_load(stg_lbm *h, const void *host, size_t bytes)
{
    const Range range("stg_lbm_load");
    if (!h || !host) return fail(h, STG_ERR_INVALID, "NULL argument");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; remove it first");
    if (bytes != ckpt_bytes(h)) return fail(h, STG_ERR_INVALID, "checkpoint size mismatch");
    CkptHeader hd{};
    std::memcpy(&hd, host, sizeof hd);
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.nx != h->d.nx || hd.ny != h->d.ny || hd.nz != h->d.nz ||
        hd.storage != h->d.storage || hd.t < 0 || hd.t0_stats < 0 || hd.t0_stats > hd.t || hd.t0_filter < 0 ||
        hd.t0_filter > hd.t || hd.streaming != h->d.streaming)
        return fail(h, STG_ERR_INVALID, "checkpoint does not match this lattice");
    int rc = wait_stream(h);
    if (rc) return rc;
    rc = reset_counters(h, hd.t);
    if (rc) return rc;
    const char *p = static_cast<const char *>(host) + sizeof hd;
    CK(cudaMemcpy(h->lat[hd.t & 1], p, hd.pop_bytes, cudaMemcpyHostToDevice));
    p += hd.pop_bytes;
    CK(cudaMemcpy(h->uf, p, hd.uf_bytes, cudaMemcpyHostToDevice));
    p += hd.uf_bytes;
    CK(cudaMemcpy(ubc_plane(h, (int)(hd.t & 1)), p, hd.plane_bytes, cudaMemcpyHostToDevice));
    p += hd.plane_bytes;
    const size_t m = (size_t)h->d.nx * h->d.ny;
    CK(cudaMemcpy(h->stat_mean, p, sizeof(double) * 3 * m, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->stat_rey, p + sizeof(double) * 3 * m, sizeof(double) * 6 * m, cudaMemcpyHostToDevice));
    StepCtl c{};
    c.t[hd.t & 1] = hd.t;
    c.t[(hd.t + 1) & 1] = hd.t;
    c.t0_filter = hd.t0_filter;
    CK(cudaMemcpy(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice));
    h->t0_stats = hd.t0_stats;
    h->mass0 = hd.mass0;
    return STG_OK;
}

int stg_lbm_get_block(stg_lbm *h, int32_t x0, int32_t y0, int32_t z0, int32_t bx, int32_t by, int32_t bz, void *host)
{
    if (!h || !host) return fail(h, STG_ERR_INVALID, "NULL argument");
    if (bx < 1 || by < 1 || bz < 1 || x0 < 0 || y0 < 0 || z0 < 0 || x0 + bx > h->d.nx || y0 + by > h->d.ny ||
        z0 + bz > h->d.nz)
        return fail(h, STG_ERR_INVALID, "block outside the lattice");
    int rc = wait_stream(h);
    if (rc) return rc;
    if (h->aa) {
        // in place: gather the canonical populations on the device, then one copy
        const size_t bytes = (size_t)19 * bx * by * bz * h->elem;
        void *tmp = nullptr;
        CK(cudaMalloc(&tmp, bytes));
        cudaError_t e = stg::launch_gather_block(h->lat[0], h->d.storage, lattice_view(h), x0, y0, z0, bx, by, bz, tmp,
                                                 h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return cuda_fail(h, e, "in-place block gather");
        return STG_OK;
    }
    // one 3-D copy per population: rows of bx elements
    for (int i = 0; i < 19; ++i) {
        cudaMemcpy3DParms m{};
        char *base = static_cast<char *>(h->lat[h->t & 1]) + (size_t)i * h->P * h->elem;
        m.srcPtr = make_cudaPitchedPtr(base, (size_t)h->d.nx * h->elem, (size_t)h->d.nx, (size_t)h->d.ny);
        m.srcPos = make_cudaPos((size_t)x0 * h->elem, (size_t)y0, (size_t)z0);
        char *dst = static_cast<char *>(host) + (size_t)i * bx * by * bz * h->elem;
        m.dstPtr = make_cudaPitchedPtr(dst, (size_t)bx * h->elem, (size_t)bx, (size_t)by);
        m.extent = make_cudaExtent((size_t)bx * h->elem, (size_t)by, (size_t)bz);
        m.kind = cudaMemcpyDeviceToHost;
        CK(cudaMemcpy3DAsync(&m, h->stream));
    }
    return wait_stream(h);
}

int stg_lbm_get_inlet(stg_lbm *h, float *host_u)
{
    if (!h || !host_u) return fail(h, STG_ERR_INVALID, "NULL argument");
    int rc = wait_stream(h);
    if (rc) return rc;
    // the plane of the last completed step
    CK(cudaMemcpy(host_u, ubc_plane(h, (int)((h->t + 1) & 1)), sizeof(float) * 3 * (size_t)h->d.ny * h->d.nz,
                  cudaMemcpyDeviceToHost));
    return STG_OK;
}

int stg_lbm_device_state(stg_lbm *h, void **pops, float **inlet_u)
{
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (pops) *pops = h->lat[h->t & 1];
    if (inlet_u) *inlet_u = ubc_plane(h, (int)((h->t + 1) & 1));
    return STG_OK;
}

int stg_lbm_info(const stg_lbm *h, stg_info *out)
{
    if (!h || !out) return STG_ERR_INVALID;
    *out = h->info;
    return STG_OK;
}

int stg_lbm_set_tile(stg_lbm *h, const stg_tile *tile)
{
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; set the batch's tile");
    if (!tile) return fail(h, STG_ERR_INVALID, "tile is NULL");
    return apply_tile(h, *tile);
}

int stg_lbm_set_probes(stg_lbm *h, int32_t n, const int32_t *xyz)
{
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (n < 0 || n > (1 << 20) || (n > 0 && !xyz)) return fail(h, STG_ERR_INVALID, "probes: 0 <= n <= 2^20");
    for (int32_t k = 0; k < n; ++k)
        if (xyz[3 * k] < 0 || xyz[3 * k] >= h->d.nx || xyz[3 * k + 1] < 0 || xyz[3 * k + 1] >= h->d.ny ||
            xyz[3 * k + 2] < 0 || xyz[3 * k + 2] >= h->d.nz)
            return fail(h, STG_ERR_INVALID, "probe outside the lattice");
    int rc = wait_stream(h);
    if (rc) return rc;
    if (n > h->n_probes || !h->probe_xyz) {
        h->probe_xyz = (int *)dalloc(h, sizeof(int) * 3 * (size_t)std::max(n, 1));
        if (!h->probe_xyz) return fail(h, STG_ERR_NOMEM, "probe table");
    }
    if (n > 0) CK(cudaMemcpy(h->probe_xyz, xyz, sizeof(int) * 3 * (size_t)n, cudaMemcpyHostToDevice));
    h->n_probes = n;
    return STG_OK;
}

int stg_lbm_step_probed(stg_lbm *h, int64_t n, float *u_host)
{
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; step the batch");
    if (n < 1 || n > 65536 || !u_host) return fail(h, STG_ERR_INVALID, "step_probed needs 1 <= n <= 65536 and a buffer");
    if (h->n_probes < 1) return fail(h, STG_ERR_INVALID, "no probes set");
    int rc = poll_check(h);
    if (rc) return rc;
    if (h->sticky) return fail(h, h->sticky, "an earlier check failed; reset the state first");
    const size_t need = (size_t)n * h->n_probes * 3;
    if (need > h->probe_cap) {
        h->probe_buf = (float *)dalloc(h, sizeof(float) * need);
        if (!h->probe_buf) {
            h->probe_cap = 0;
            return fail(h, STG_ERR_NOMEM, "probe buffer");
        }
        h->probe_cap = need;
    }
    const int64_t t_before = h->t;
    for (int64_t s = 0; s < n; ++s) {
        CK(cudaGraphLaunch(h->g_single[h->t & 1][is_stats_step(h, h->t) ? 1 : 0], h->stream));
        h->t += 1;
        CK(stg::launch_probe(h->lat[h->t & 1], h->d.storage, lattice_view(h), h->n_probes, h->probe_xyz,
                             (float)h->d.force[0], (float)h->d.force[1], (float)h->d.force[2],
                             h->probe_buf + (size_t)s * h->n_probes * 3, h->stream));
    }
    rc = queue_check_readback(h, t_before);
    if (rc) return rc;
    CK(cudaMemcpyAsync(u_host, h->probe_buf, sizeof(float) * need, cudaMemcpyDeviceToHost, h->stream));
    return wait_stream(h);
}

int stg_lbm_get_tile(const stg_lbm *h, stg_tile *tile)
{
    if (!h || !tile) return STG_ERR_INVALID;
    *tile = h->tile;
    return STG_OK;
}

}  // extern "C"

namespace stg {
namespace host {

cudaError_t trial_pass(stg_lbm *h, const stg_tile &tile, cudaStream_t s, int k)
{
    const int parity = (int)((h->t + (h->aa ? k : 0)) & 1);
    const stg_tile keep = h->tile;
    h->tile = tile;
    stg::StepArgs a = step_args(h, parity);
    h->tile = keep;
    a.stats_every = 0;  // the edge kernel samples on its own otherwise
    return stg::launch_step(a, h->d.storage, h->d.collision, false, s, h->side, h->ev_fork, h->ev_join);
}

int save_trial_state(stg_lbm *h, std::vector<unsigned char> &pops, stg::StepCtl &ctl)
{
    if (!h->aa) return STG_OK;
    int rc = wait_stream(h);
    if (rc) return rc;
    pops.resize(19 * h->P * h->elem);
    CK(cudaMemcpy(pops.data(), h->lat[0], pops.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&ctl, h->ctl, sizeof ctl, cudaMemcpyDeviceToHost));
    return STG_OK;
}

int restore_trial_state(stg_lbm *h, const std::vector<unsigned char> &pops, const stg::StepCtl &ctl)
{
    if (!h->aa) return STG_OK;
    int rc = wait_stream(h);
    if (rc) return rc;
    CK(cudaMemcpy(h->lat[0], pops.data(), pops.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice));
    return STG_OK;
}

int apply_tile(stg_lbm *h, const stg_tile &tile)
{
    if (!tile_ok(tile)) return fail(h, STG_ERR_INVALID, "tile: layout 0 or 1, z chunks 0 or >= 4");
    int rc = wait_stream(h);
    if (rc) return rc;
    const stg_tile old = h->tile;
    h->tile = tile;
    h->tile.pad0 = 0;
    rc = capture_all(h);
    if (rc) {
        h->tile = old;
        capture_all(h);
    }
    return rc;
}

const stg_tile *tile_candidates(int *n)
{
    static const stg_tile cand[] = {{1, 4, 24, 0},  {1, 6, 24, 0},  {1, 8, 24, 0},  {1, 12, 24, 0}, {1, 16, 24, 0},
                                    {1, 8, 8, 0},   {0, 16, 24, 0}, {0, 24, 24, 0}, {0, 48, 24, 0}, {0, 0, 0, 0}};
    *n = (int)(sizeof cand / sizeof cand[0]);
    return cand;
}

}  // namespace host
}  // namespace stg

extern "C" {

int stg_lbm_autotune(stg_lbm *h, int32_t trial_passes, stg_tile *chosen)
{
    const Range range("stg_lbm_autotune");
    if (!h) return fail(nullptr, STG_ERR_INVALID, "handle is NULL");
    if (h->batch) return fail(h, STG_ERR_INVALID, "the lattice is in a batch; tune the batch");
    if (trial_passes < 1 || trial_passes > 1000) return fail(h, STG_ERR_INVALID, "trial_passes must be in [1, 1000]");
    if (h->sticky) return fail(h, h->sticky, "an earlier check failed; reset the state first");
    int ncand = 0;
    const stg_tile *cand = tile_candidates(&ncand);
    int rc = wait_stream(h);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(h, STG_ERR_CUDA, "cudaEventCreate");
    }
    // plain passes from the current state: src = lat[t & 1], dst = lat[(t & 1) ^ 1];
    // the pass writes the device counter t[p ^ 1] = t + 1, which the next real
    // step writes again, and the mass slots, which every pass rewrites.  In
    // place the passes update the lattice, which is saved first and put back.
    std::vector<unsigned char> keep;
    StepCtl keep_ctl{};
    rc = save_trial_state(h, keep, keep_ctl);
    stg_tile best = h->tile;
    float best_ms = -1.f;
    for (int c = 0; c < ncand && rc == STG_OK; ++c) {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k <= trial_passes && e == cudaSuccess; ++k) {
            if (k == 1) e = cudaEventRecord(e0, h->stream);
            if (e == cudaSuccess) e = trial_pass(h, cand[c], h->stream, k);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "autotune pass");
        else if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc2 = restore_trial_state(h, keep, keep_ctl);
    if (rc) return rc;
    if (rc2) return rc2;
    rc = apply_tile(h, best);
    if (rc == STG_OK && chosen) *chosen = best;
    return rc;
}

void stg_lbm_destroy(stg_lbm *h) { release(h); }

const char *stg_lbm_last_error(const stg_lbm *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

int stg_mode_draws(uint64_t seed, int32_t n, double *out)
{
    if (n < 0 || (n > 0 && !out)) return STG_ERR_INVALID;
    splitmix_uniform(seed, 4 * n, out);
    return STG_OK;
}

const char *stg_lbm_version(void) { return "stglbm 0.1 (sm_103a)"; }

}  // extern "C"
