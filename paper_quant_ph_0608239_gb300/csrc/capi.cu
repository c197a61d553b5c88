// capi.cu -- the extern "C" boundary declared in include/qsim.h: handles,
// argument checks, the qubit-to-bit map sigma (Sec. III.B), dispatch of gates
// to the sweep and tile kernels, reductions and host transfers.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <thread>
#include <atomic>

#include <cuda_runtime.h>

#include "../../include/qsim.h"
#include "kernels.hpp"
#include "planner.hpp"

using namespace qsim;

// ----------------------------------------------------------------- errors
static thread_local std::string g_err;

static qsim_status fail(qsim_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

static qsim_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? QSIM_ENOMEM : QSIM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ----------------------------------------------------------------- handle
struct ProfRec {
    int fam;
    cudaEvent_t a, b;
    double bytes, flops;
};

struct qsim_state {
    int n = 0;
    qsim_dtype dt = QSIM_C64;
    void *amp = nullptr;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 152;
    int phys[64];              // logical qubit q -> index bit
    double *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    double *d_res = nullptr;   // small device result area (64 doubles)
    double *h_res = nullptr;   // pinned host mirror
    uint32_t *d_err = nullptr; // bounded-wait error word
    TileOp *d_ops = nullptr;
    size_t ops_cap = 0;
    void *d_dense = nullptr;   // dense matrices (state precision)
    size_t dense_cap = 0;
    void *d_chunk = nullptr;   // staging for logical-order reads
    size_t chunk_bytes = 0;
    TileOp *h_ops = nullptr;   // pinned staging of gate programs
    size_t h_ops_cap = 0;
    TilePhase *d_phases = nullptr;
    size_t phases_cap = 0;
    TilePhase *h_phases = nullptr;
    size_t h_phases_cap = 0;
    cudaEvent_t upload_done = nullptr;
    // instrumentation
    bool prof = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    uint64_t launches = 0, h2d = 0, d2h = 0;
};

// Kernel families reported by qsim_profile_read.
enum Fam { F_INIT, F_PAIR, F_DIAG, F_DENSE, F_TILE, F_NORM, F_BITS, F_PROBS, F_GATHER, F_SAMPLE, F_FUSED_TC,
           F_BATCH, F_FUSED_TC128, F_FUSED_TC6, F_PERM, F_PHASE, F_COUNT };
static const char *kFamName[F_COUNT] = {"init_basis", "pair_sweep", "diag_sweep", "dense_cuda_core", "tile_pass",
                                        "norm", "bit_probs", "probs", "gather", "sample", "fused_tensor_core",
                                        "batch", "fused_tc_digits", "fused_tc_bf16x3", "interchange",
                                        "phase_pass"};

static cudaEvent_t take_event(qsim_state *h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Every kernel launch made for a handle goes through here: it is counted and,
// when profiling is on, bracketed by events on the handle's stream.
template <class F>
static cudaError_t launch(qsim_state *h, int fam, double alg_bytes, int nkernels, F &&f, double alg_flops = 0.0) {
    h->launches += (uint64_t)nkernels;
    if (!h->prof) return f();
    cudaEvent_t a = take_event(h), b = take_event(h);
    cudaEventRecord(a, h->stream);
    cudaError_t e = f();
    cudaEventRecord(b, h->stream);
    h->recs.push_back(ProfRec{fam, a, b, alg_bytes, alg_flops});
    return e;
}

static size_t amp_bytes(qsim_dtype dt) { return dt == QSIM_C64 ? 8 : 16; }
static size_t state_bytes(const qsim_state *h) { return amp_bytes(h->dt) << h->n; }
static bool identity_layout(const qsim_state *h) {
    for (int q = 0; q < h->n; q++)
        if (h->phys[q] != q) return false;
    return true;
}

static qsim_status init_common(qsim_state *h) {
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    CK(cudaGetDevice(&h->device), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device), "device attribute");
    h->scratch_bytes = std::max(reduce_scratch_bytes(h->n), (size_t)4096);
    CK(cudaMalloc(&h->d_scratch, h->scratch_bytes), "cudaMalloc scratch");
    CK(cudaMalloc(&h->d_res, 64 * sizeof(double)), "cudaMalloc results");
    CK(cudaMallocHost(&h->h_res, 64 * sizeof(double)), "cudaMallocHost results");
    CK(cudaMalloc(&h->d_err, sizeof(uint32_t)), "cudaMalloc error word");
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream), "memset error word");
    return QSIM_OK;
}

static void release(qsim_state *h) {
    if (!h) return;
    for (auto &r : h->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    if (h->upload_done) cudaEventDestroy(h->upload_done);
    if (h->h_ops) cudaFreeHost(h->h_ops);
    if (h->h_phases) cudaFreeHost(h->h_phases);
    if (h->d_phases) cudaFree(h->d_phases);
    if (h->owns && h->amp) cudaFree(h->amp);
    if (h->d_scratch) cudaFree(h->d_scratch);
    if (h->d_res) cudaFree(h->d_res);
    if (h->h_res) cudaFreeHost(h->h_res);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_ops) cudaFree(h->d_ops);
    if (h->d_dense) cudaFree(h->d_dense);
    if (h->d_chunk) cudaFree(h->d_chunk);
    delete h;
}

// Wait for the stream and turn a device-side timeout into ETIMEOUT.
static qsim_status sync_check(qsim_state *h) {
    CK(cudaMemcpyAsync(h->h_res + 63, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream),
       "read error word");
    h->d2h += sizeof(uint32_t);
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    uint32_t e;
    std::memcpy(&e, h->h_res + 63, sizeof e);
    if (e != 0) {
        cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream);
        cudaStreamSynchronize(h->stream);
        return fail(QSIM_ETIMEOUT, "a bounded device-side wait expired (code %u)", e);
    }
    return QSIM_OK;
}

#define CHECK_HANDLE(h) \
    if (!(h)) return fail(QSIM_EINVAL, "null handle")

extern "C" {

const char *qsim_last_error(void) { return g_err.c_str(); }

const char *qsim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

void qsim_default_opts(qsim_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->mode = QSIM_MODE_FUSED;
}

qsim_status qsim_alloc(int n, qsim_dtype dt, qsim_handle *out) {
    if (!out) return fail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(QSIM_EINVAL, "n = %d outside [1, %d]", n, kMaxQubits);
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_EINVAL, "bad dtype %d", (int)dt);
    qsim_state *h = new qsim_state;
    h->n = n;
    h->dt = dt;
    h->owns = true;
    cudaError_t e = cudaMalloc(&h->amp, state_bytes(h));
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->amp = nullptr;
        release(h);
        return cuda_fail(e, "cudaMalloc state");
    }
    qsim_status st = init_common(h);
    if (st == QSIM_OK) {
        e = launch(h, F_INIT, (double)state_bytes(h), 1,
                   [&] { return launch_init_basis(h->amp, (int)dt, n, 0, h->stream); });
        if (e != cudaSuccess) st = cuda_fail(e, "init basis");
    }
    if (st != QSIM_OK) {
        release(h);
        return st;
    }
    *out = h;
    return QSIM_OK;
}

qsim_status qsim_attach(void *dev_ptr, int n, qsim_dtype dt, void *stream, qsim_handle *out) {
    if (!out) return fail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 15u))
        return fail(QSIM_EINVAL, "device pointer must be non-NULL and 16-byte aligned");
    if (n < 1 || n > kMaxQubits) return fail(QSIM_EINVAL, "n = %d outside [1, %d]", n, kMaxQubits);
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_EINVAL, "bad dtype %d", (int)dt);
    qsim_state *h = new qsim_state;
    h->n = n;
    h->dt = dt;
    h->amp = dev_ptr;
    h->owns = false;
    h->stream = static_cast<cudaStream_t>(stream);
    qsim_status st = init_common(h);
    if (st != QSIM_OK) {
        release(h);
        return st;
    }
    *out = h;
    return QSIM_OK;
}

qsim_status qsim_free(qsim_handle h) {
    if (!h) return QSIM_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    return QSIM_OK;
}

qsim_status qsim_set_stream(qsim_handle h, void *s) {
    CHECK_HANDLE(h);
    h->stream = static_cast<cudaStream_t>(s);
    return QSIM_OK;
}

qsim_status qsim_info(qsim_handle h, int *n, qsim_dtype *dt, void **dev_ptr) {
    CHECK_HANDLE(h);
    if (n) *n = h->n;
    if (dt) *dt = h->dt;
    if (dev_ptr) *dev_ptr = h->amp;
    return QSIM_OK;
}

qsim_status qsim_set_basis(qsim_handle h, uint64_t x) {
    CHECK_HANDLE(h);
    if (h->n < 64 && x >= (1ull << h->n)) return fail(QSIM_EINVAL, "basis index out of range");
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    CK(launch(h, F_INIT, (double)state_bytes(h), 1,
              [&] { return launch_init_basis(h->amp, (int)h->dt, h->n, x, h->stream); }),
       "init basis");
    return QSIM_OK;
}

qsim_status qsim_set_shor_state(qsim_handle h, int X, uint64_t y, uint64_t G) {
    CHECK_HANDLE(h);
    if (X < 1 || X >= h->n) return fail(QSIM_EINVAL, "X = %d outside [1, n)", X);
    if (G < 2 || G >= (1ull << 32) || G > (1ull << (h->n - X)))
        return fail(QSIM_EINVAL, "G = %llu: need 2 <= G <= 2^(n - X) and G < 2^32", (unsigned long long)G);
    if (y < 1 || y >= G) return fail(QSIM_EINVAL, "y must lie in [1, G)");
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    CK(launch(h, F_INIT, (double)state_bytes(h), 1,
              [&] { return launch_shor_state(h->amp, (int)h->dt, h->n, X, y, G, h->stream); }),
       "Shor initial state");
    return QSIM_OK;
}

qsim_status qsim_set_state(qsim_handle h, const void *host_in, size_t bytes) {
    CHECK_HANDLE(h);
    if (!host_in || bytes != state_bytes(h)) return fail(QSIM_EINVAL, "need %zu bytes", state_bytes(h));
    for (int q = 0; q < 64; q++) h->phys[q] = q;
    CK(cudaMemcpyAsync(h->amp, host_in, bytes, cudaMemcpyHostToDevice, h->stream), "copy state in");
    h->h2d += bytes;
    CK(cudaStreamSynchronize(h->stream), "sync");
    return QSIM_OK;
}

// ------------------------------------------------------------------ gates
static qsim_status sweep_gate(qsim_state *h, const PGate &pg) {
    FixedBitsHost fb{};
    uint64_t pmask;
    bool single;
    fixed_bits_for(pg, fb, pmask, single);
    if (fb.npos > h->n) return QSIM_OK;  // cannot happen after validation
    const double touched = std::ldexp(single ? 1.0 : 2.0, h->n - fb.npos);
    const double bytes = 2.0 * (double)amp_bytes(h->dt) * touched;
    const double flops = gate_flops(pg, h->n);
    cudaError_t e = single ? launch(h, F_DIAG, bytes, 1,
                                    [&] { return launch_diag(h->amp, (int)h->dt, h->n, fb, pg.t0, pg.U, h->stream); },
                                    flops)
                           : launch(h, F_PAIR, bytes, 1, [&] {
                                 return launch_pairs(h->amp, (int)h->dt, h->n, fb, pmask, pg.gc, pg.U, h->stream);
                             }, flops);
    if (e != cudaSuccess) return cuda_fail(e, "gate sweep");
    return QSIM_OK;
}

static qsim_status apply_u(qsim_state *h, uint64_t ctrl, int t, const double U[8]) {
    if (!U) return fail(QSIM_EINVAL, "U is NULL");
    qsim_gate g{};
    g.kind = QSIM_GATE_U;
    g.target = t;
    g.ctrl_mask = ctrl;
    for (int k = 0; k < 8; k++) g.param[k] = U[k];
    PGate pg;
    std::string msg;
    if (!prepare_gate(g, h->n, h->phys, pg, msg)) return fail(QSIM_EINVAL, "%s", msg.c_str());
    return sweep_gate(h, pg);
}

qsim_status qsim_apply_1q(qsim_handle h, int t, const double U[8]) {
    CHECK_HANDLE(h);
    return apply_u(h, 0, t, U);
}

qsim_status qsim_apply_ctrl(qsim_handle h, uint64_t ctrl_mask, int t, const double U[8]) {
    CHECK_HANDLE(h);
    return apply_u(h, ctrl_mask, t, U);
}

qsim_status qsim_apply_gate(qsim_handle h, const qsim_gate *g) {
    CHECK_HANDLE(h);
    if (!g) return fail(QSIM_EINVAL, "gate is NULL");
    PGate pg;
    std::string msg;
    if (!prepare_gate(*g, h->n, h->phys, pg, msg)) return fail(QSIM_EINVAL, "%s", msg.c_str());
    return sweep_gate(h, pg);
}

// Tile shape: the register-blocked kernel takes T = 12 (or 13 for
// complex64) when n >= T; other tile sizes use the shared-memory kernel.
static void tile_defaults(const qsim_state *h, const qsim_opts *o, int &T, int &L, int &RB) {
    T = (o && o->tile_bits > 0) ? o->tile_bits : 12;
    const int Tmax = 13;
    if (T > Tmax) T = Tmax;
    if (T < 2) T = 2;
    RB = (tile2_supported((int)h->dt, T) && h->n >= T) ? T - 5 - kRegWarpBits : 0;
    L = RB ? 5 : (h->dt == QSIM_C64 ? 5 : 4);
    if (T - L > 10) L = T - 10;
    if (L >= T) L = T - 2;
    if (L < 1) L = 1;
}

}  // extern "C"

template <class T>
static qsim_status stage(qsim_state *h, const std::vector<T> &v, T *&dbuf, size_t &dcap, T *&hbuf, size_t &hcap,
                         const char *what) {
    if (v.empty()) return QSIM_OK;
    if (v.size() > dcap) {
        if (dbuf) {
            CK(cudaStreamSynchronize(h->stream), "sync before regrow");
            cudaFree(dbuf);
            dbuf = nullptr;
            dcap = 0;
        }
        const size_t cap = std::max(v.size(), (size_t)256);
        CK(cudaMalloc(&dbuf, cap * sizeof(T)), what);
        dcap = cap;
    }
    if (v.size() > hcap) {
        if (hbuf) cudaFreeHost(hbuf);
        hbuf = nullptr;
        hcap = 0;
        const size_t cap = std::max(v.size(), (size_t)1024);
        CK(cudaMallocHost(&hbuf, cap * sizeof(T)), "cudaMallocHost staging");
        hcap = cap;
    }
    std::memcpy(hbuf, v.data(), v.size() * sizeof(T));
    CK(cudaMemcpyAsync(dbuf, hbuf, v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream), what);
    h->h2d += v.size() * sizeof(T);
    return QSIM_OK;
}

extern "C" {

static qsim_status ensure_dense(qsim_state *h, size_t bytes) {
    if (bytes <= h->dense_cap) return QSIM_OK;
    if (h->d_dense) {
        CK(cudaStreamSynchronize(h->stream), "sync");
        cudaFree(h->d_dense);
        h->d_dense = nullptr;
        h->dense_cap = 0;
    }
    const size_t cap = std::max(bytes, (size_t)65536);
    CK(cudaMalloc(&h->d_dense, cap), "cudaMalloc dense");
    h->dense_cap = cap;
    return QSIM_OK;
}

static qsim_status upload_program(qsim_state *h, const Plan &plan) {
    if (!h->upload_done) CK(cudaEventCreateWithFlags(&h->upload_done, cudaEventDisableTiming), "event");
    CK(cudaEventSynchronize(h->upload_done), "wait staging");
    qsim_status st = stage(h, plan.ops, h->d_ops, h->ops_cap, h->h_ops, h->h_ops_cap, "upload tile ops");
    if (st != QSIM_OK) return st;
    st = stage(h, plan.phases, h->d_phases, h->phases_cap, h->h_phases, h->h_phases_cap, "upload tile phases");
    if (st != QSIM_OK) return st;
    CK(cudaEventRecord(h->upload_done, h->stream), "event record");
    return QSIM_OK;
}

static qsim_status launch_passes(qsim_state *h, const Plan &plan, const TileOp *d_ops, const TilePhase *d_phases) {
    const double pass_bytes = 2.0 * (double)state_bytes(h);
    // complex128: the state stays in double-float form in HBM from the first
    // arithmetic pass to the last one of this run (only those two convert);
    // every pass of a complex128 plan runs in k_tile_df.  A run that fails
    // part-way leaves the state unspecified, as any failed run does.
    int last_arith = -1;
    bool df_carry = h->dt == QSIM_C128;
    for (size_t i = 0; i < plan.passes.size(); i++) {
        const PassPlan &pp = plan.passes[i];
        if (pp.phase_count > 0) df_carry = false;
        if (pp.phase_count == 0 && pp.op_count > 0 && pp.arith) last_arith = (int)i;
    }
    bool in_df = false;  // the state is in double-float form now
    for (size_t pi = 0; pi < plan.passes.size(); pi++) {
        const PassPlan &pp = plan.passes[pi];
        if (pp.phase_count > 0) {
            CK(launch(h, F_TILE, pass_bytes, 1,
                      [&] {
                          return launch_tile_pass2(h->amp, (int)h->dt, pp.geom, d_phases + pp.phase_begin,
                                                   pp.phase_count, d_ops, pp.op_begin, pp.op_count, h->d_err,
                                                   h->sm_count, h->stream);
                      },
                      pp.flops),
               "register tile pass");
            continue;
        }
        if (pp.op_count == 0) continue;
        if (h->dt == QSIM_C128) {
            const bool cvt_in = pp.arith && !in_df;
            const bool cvt_out = pp.arith && (!df_carry || (int)pi == last_arith);
            CK(launch(h, F_TILE, pass_bytes, 1,
                      [&] {
                          return launch_tile_pass_df(h->amp, pp.geom, d_ops + pp.op_begin, pp.op_count - pp.nglob,
                                                     pp.nglob, pp.absorber, cvt_in, cvt_out, h->d_err, h->sm_count,
                                                     h->stream);
                      },
                      pp.flops),
               "double-float tile pass");
            if (pp.arith) in_df = !cvt_out;
            continue;
        }
        CK(launch(h, F_TILE, pass_bytes, 1,
                  [&] {
                      return launch_tile_pass(h->amp, (int)h->dt, pp.geom, d_ops + pp.op_begin, pp.op_count,
                                              h->d_dense, h->d_err, h->sm_count, h->stream);
                  },
                  pp.flops),
           "tile pass");
    }
    return QSIM_OK;
}

static qsim_status prepare_all(qsim_state *h, const qsim_gate *gates, size_t ng, std::vector<PGate> &out) {
    out.resize(ng);
    std::string msg;
    for (size_t i = 0; i < ng; i++)
        if (!prepare_gate(gates[i], h->n, h->phys, out[i], msg))
            return fail(QSIM_EINVAL, "gate %zu: %s", i, msg.c_str());
    return QSIM_OK;
}

// A planned circuit.
struct qsim_plan_s {
    int n = 0;
    qsim_dtype dt = QSIM_C64;
    int phys[64];
    int mode = QSIM_MODE_FUSED;
    std::vector<PGate> sweeps;   // PERGATE mode
    Plan plan;                   // FUSED mode
    TileOp *d_ops = nullptr;
    TilePhase *d_phases = nullptr;
    std::vector<FusedBlock> blocks;  // FUSED mode with fuse_k: dense blocks on the tensor cores
    std::vector<float> bmats;        // their B operands, 2 (2^(k+1))^2 floats each
    float *d_bmats = nullptr;
    // dense blocks the tensor-core kernel does not take (complex128, k = 6, ...)
    // run on the CUDA cores (k_dense): their matrices in the state's precision
    bool cuda_core = false;
    bool tc128 = false;  // complex128 blocks on the tensor cores (bmats holds bf16 slices)
    bool tc6 = false;    // complex64 6-qubit blocks on the tensor cores (bmats holds bf16 slices)
    std::vector<unsigned char> cmats;
    size_t cmat_stride = 0;
    void *d_cmats = nullptr;
    // runs of commuting phase shifts among the dense blocks (tensor-core
    // plans): their tables, concatenated
    std::vector<PhasePass> phases;
    std::vector<uint32_t> phase_words;
    std::vector<size_t> phase_off;  // word offset of each pass's tables
    uint32_t *d_phase = nullptr;
    qsim_plan_stats stats{};
    // QSIM_MODE_AUTO: one candidate plan per tile size / fusion width; the
    // first runs time each candidate, later runs use the fastest
    std::vector<qsim_plan_s *> cands;
    std::vector<cudaEvent_t> ev;  // start, end per candidate
    int next = 0;
    int chosen = -1;
};

// Runs of at least this many commuting phase shifts over more than k qubits
// may become one phase pass (planner.hpp, plan_fused_phases).
constexpr int kPhaseRunMin = 24;
// complex128 phase passes hold 64-bit tables in shared memory: at most 24
constexpr int kMaxPhaseTables128 = 24;

// The phase passes' tables for the device: complex64 passes take the top 32
// bits of each 64-bit entry (rounded), complex128 ones the whole entry (two
// 32-bit words, low first).
static void gather_phase_tables(qsim_plan_s &P, bool wide) {
    P.phase_words.clear();
    P.phase_off.clear();
    for (const PhasePass &pp : P.phases) {
        P.phase_off.push_back(P.phase_words.size());
        for (uint64_t w : pp.words) {
            if (wide) {
                P.phase_words.push_back((uint32_t)w);
                P.phase_words.push_back((uint32_t)(w >> 32));
            } else {
                P.phase_words.push_back((uint32_t)((w + (1ull << 31)) >> 32));
            }
        }
    }
}

// search: the block planner also tries its beam search (plan_fused); the
// batch's many small plans skip it
static qsim_status build_plan(qsim_state *h, const qsim_gate *gates, size_t ng, const qsim_opts *opts,
                              qsim_plan_s &P, bool search = true) {
    if (ng && !gates) return fail(QSIM_EINVAL, "gates is NULL");
    qsim_opts o;
    qsim_default_opts(&o);
    if (opts) o = *opts;
    if (o.mode == QSIM_MODE_AUTO) o.mode = QSIM_MODE_FUSED;  // a single run cannot time candidates
    if (o.mode != QSIM_MODE_FUSED && o.mode != QSIM_MODE_PERGATE) return fail(QSIM_EINVAL, "unknown mode %d", o.mode);
    std::vector<PGate> pg;
    qsim_status st = prepare_all(h, gates, ng, pg);
    if (st != QSIM_OK) return st;
    P.n = h->n;
    P.dt = h->dt;
    std::memcpy(P.phys, h->phys, sizeof P.phys);
    P.mode = o.mode;
    P.stats = qsim_plan_stats{};
    P.stats.gates = (double)ng;
    if (o.mode == QSIM_MODE_PERGATE) {
        P.sweeps = std::move(pg);
        P.stats.sweeps = (int)P.sweeps.size();
        for (const PGate &g : P.sweeps) {
            FixedBitsHost fb{};
            uint64_t pmask;
            bool single;
            fixed_bits_for(g, fb, pmask, single);
            P.stats.alg_bytes += 2.0 * (double)amp_bytes(h->dt) * std::ldexp(single ? 1.0 : 2.0, h->n - fb.npos);
            P.stats.alg_flops += gate_flops(g, h->n);
        }
        return QSIM_OK;
    }
    if (o.fuse_k > 0 && h->dt == QSIM_C128 && fused_tc128_supported(o.fuse_k, h->n)) {
        // complex128 blocks on the tensor cores (bf16 digit slices) and phase
        // passes; a block the scheme cannot take exactly sends the whole plan
        // to the CUDA cores
        if (!plan_fused_phases(pg, h->n, o.fuse_k, kPhaseRunMin, kMaxPhaseTables128, P.blocks, P.phases, search))
            return fail(QSIM_EINVAL, "a gate acts on more qubits than fuse_k");
        gather_phase_tables(P, true);
        const size_t per = fused_tc128_b_bytes() / sizeof(float);
        P.bmats.resize(per * P.blocks.size());
        bool ok = true;
        for (size_t b = 0; b < P.blocks.size() && ok; b++) {
            if (P.blocks[b].phase >= 0) {
                P.stats.alg_flops += P.blocks[b].flops;
                continue;
            }
            TileGeom g;
            FusedMap fm;
            ok = fused_geometry(h->n, o.fuse_k, P.blocks[b].pos, g, fm) &&
                 fused_tc128_prepare_b(P.blocks[b].U.data(), reinterpret_cast<uint16_t *>(P.bmats.data() + per * b));
            P.stats.alg_flops += P.blocks[b].flops;
        }
        if (ok) {
            P.tc128 = true;
            P.stats.passes = (int)P.blocks.size();
            P.stats.tile_bits = o.fuse_k + 7;
            P.stats.alg_bytes = 2.0 * (double)state_bytes(h) * P.stats.passes;
            return QSIM_OK;
        }
        P.blocks.clear();
        P.bmats.clear();
        P.phases.clear();
        P.phase_words.clear();
        P.phase_off.clear();
        P.stats.alg_flops = 0.0;
    }
    if (o.fuse_k == 6 && h->dt == QSIM_C64 && fused_tc6_supported(h->n)) {
        // complex64 6-qubit blocks on the tensor cores (bf16 hi/mid/lo slices),
        // long runs of phase shifts as phase passes
        if (!plan_fused_phases(pg, h->n, o.fuse_k, kPhaseRunMin, kMaxPhaseTables, P.blocks, P.phases, search))
            return fail(QSIM_EINVAL, "a gate acts on more qubits than fuse_k");
        gather_phase_tables(P, false);
        const size_t per = fused_tc6_b_bytes() / sizeof(float);
        P.bmats.resize(per * P.blocks.size());
        for (size_t b = 0; b < P.blocks.size(); b++) {
            if (P.blocks[b].phase >= 0) {
                P.stats.alg_flops += P.blocks[b].flops;
                continue;
            }
            TileGeom g;
            FusedMap fm;
            if (!fused_geometry(h->n, o.fuse_k, P.blocks[b].pos, g, fm))
                return fail(QSIM_EUNSUPPORTED, "no tile geometry for a fused block");
            fused_tc6_prepare_b(P.blocks[b].U.data(), reinterpret_cast<uint16_t *>(P.bmats.data() + per * b));
            P.stats.alg_flops += P.blocks[b].flops;
        }
        P.tc6 = true;
        P.stats.passes = (int)P.blocks.size();
        P.stats.tile_bits = o.fuse_k + 7;
        P.stats.alg_bytes = 2.0 * (double)state_bytes(h) * P.stats.passes;
        return QSIM_OK;
    }
    if (o.fuse_k > 0 && (h->dt == QSIM_C128 || !fused_tc_supported((int)h->dt, o.fuse_k, h->n))) {
        // dense blocks on the CUDA cores (complex128, k = 1..6, small registers)
        if (o.fuse_k > 6 || o.fuse_k > h->n) return fail(QSIM_EUNSUPPORTED, "fused blocks need k <= min(6, n)");
        if (!plan_fused(pg, h->n, o.fuse_k, P.blocks, search))
            return fail(QSIM_EINVAL, "a gate acts on more qubits than fuse_k");
        const size_t ent = (size_t)1 << (2 * o.fuse_k);
        P.cuda_core = true;
        P.cmat_stride = ent * amp_bytes(h->dt);
        P.cmats.resize(P.cmat_stride * P.blocks.size());
        for (size_t b = 0; b < P.blocks.size(); b++) {
            const std::vector<double> &U = P.blocks[b].U;
            unsigned char *dst = P.cmats.data() + P.cmat_stride * b;
            if (h->dt == QSIM_C64) {
                for (size_t i = 0; i < 2 * ent; i++) {
                    const float f = (float)U[i];
                    std::memcpy(dst + 4 * i, &f, 4);
                }
            } else {
                std::memcpy(dst, U.data(), 16 * ent);
            }
            P.stats.alg_flops += P.blocks[b].flops;
        }
        P.stats.passes = (int)P.blocks.size();
        P.stats.tile_bits = 0;
        P.stats.alg_bytes = 2.0 * (double)state_bytes(h) * P.stats.passes;
        return QSIM_OK;
    }
    if (o.fuse_k > 0) {
        // complex64 4- and 5-qubit blocks on the tensor cores (3xTF32), long
        // runs of phase shifts as phase passes
        if (!plan_fused_phases(pg, h->n, o.fuse_k, kPhaseRunMin, kMaxPhaseTables, P.blocks, P.phases, search))
            return fail(QSIM_EINVAL, "a gate acts on more qubits than fuse_k");
        gather_phase_tables(P, false);
        const size_t per = 2 * (size_t)(2 << o.fuse_k) * (size_t)(2 << o.fuse_k);
        P.bmats.resize(per * P.blocks.size());
        for (size_t b = 0; b < P.blocks.size(); b++) {
            if (P.blocks[b].phase >= 0) {
                P.stats.alg_flops += P.blocks[b].flops;
                continue;
            }
            TileGeom g;
            FusedMap fm;
            if (!fused_geometry(h->n, o.fuse_k, P.blocks[b].pos, g, fm))
                return fail(QSIM_EUNSUPPORTED, "no tile geometry for a fused block");
            fused_tc_prepare_b(o.fuse_k, P.blocks[b].U.data(), P.bmats.data() + per * b);
            P.stats.alg_flops += P.blocks[b].flops;
        }
        P.stats.passes = (int)P.blocks.size();
        P.stats.tile_bits = o.fuse_k + 7;
        P.stats.alg_bytes = 2.0 * (double)state_bytes(h) * P.stats.passes;
        return QSIM_OK;
    }
    int T, L, RB;
    tile_defaults(h, &o, T, L, RB);
    // register passes stay within the staged-program capacity of k_tile2
    plan_tiles(pg, h->n, T, L, P.plan, RB, RB ? kRegMaxOps : 0, RB ? kRegMaxPhases : 0);
    if (h->dt == QSIM_C128) {
        defer_butterflies(P.plan);
        merge_local_diagonals(P.plan);
        hoist_global_diagonals(P.plan);
    }
    P.stats.ops = 0;  // (a pass shrunk by merging leaves unused entries in the op array)
    for (const PassPlan &pp : P.plan.passes) {
        if (pp.op_count || pp.phase_count) P.stats.passes++;
        P.stats.ops += pp.op_count;
    }
    P.stats.phases = (int)P.plan.phases.size();
    P.stats.tile_bits = P.plan.passes.empty() ? 0 : P.plan.passes[0].geom.L + P.plan.passes[0].geom.H;
    P.stats.alg_bytes = 2.0 * (double)state_bytes(h) * P.stats.passes;
    for (const PassPlan &pp : P.plan.passes) P.stats.alg_flops += pp.flops;
    return QSIM_OK;
}

// a phase pass among the blocks (tensor-core plans, either precision); a
// complex128 pass reads and writes IEEE doubles only as the first / last
// step of the plan, double-float form otherwise (as the blocks around it)
static qsim_status run_phase(qsim_state *h, const qsim_plan_s &P, const uint32_t *d_phase, int idx,
                             bool in_ieee = true, bool out_ieee = true) {
    const PhasePass &pp = P.phases[(size_t)idx];
    PhaseMeta m{};
    m.ntab = (int32_t)pp.ta.size();
    for (size_t t = 0; t < pp.ta.size() && t < (size_t)kMaxPhaseTables; t++) {
        m.ta[t] = pp.ta[t];
        m.tb[t] = pp.tb[t];
    }
    const uint32_t *tabs = d_phase + P.phase_off[(size_t)idx];
    CK(launch(h, F_PHASE, 2.0 * (double)state_bytes(h), 1,
              [&] {
                  return h->dt == QSIM_C64 ? launch_phase_pass(h->amp, h->n, tabs, m, h->sm_count, h->stream)
                                           : launch_phase_pass128(h->amp, h->n, reinterpret_cast<const uint64_t *>(tabs),
                                                                  m, h->sm_count, h->stream, in_ieee, out_ieee);
              },
              8.0 * std::ldexp(1.0, h->n)),
       "phase pass");
    return QSIM_OK;
}

static qsim_status run_blocks(qsim_state *h, const qsim_plan_s &P, const float *d_bmats, const void *d_cmats,
                              const uint32_t *d_phase) {
    if (P.blocks.empty()) return QSIM_OK;
    const int k = P.blocks[0].k;
    if (P.cuda_core) {
        for (size_t b = 0; b < P.blocks.size(); b++) {
            const void *dU = static_cast<const unsigned char *>(d_cmats) + P.cmat_stride * b;
            CK(launch(h, F_DENSE, 2.0 * (double)state_bytes(h), 1,
                      [&] { return launch_dense(h->amp, (int)h->dt, h->n, k, P.blocks[b].pos, dU, h->stream); },
                      P.blocks[b].flops),
               "fused block (CUDA cores)");
        }
        return QSIM_OK;
    }
    if (P.tc6) {
        const size_t per = fused_tc6_b_bytes() / sizeof(float);
        for (size_t b = 0; b < P.blocks.size(); b++) {
            if (P.blocks[b].phase >= 0) {
                const qsim_status st = run_phase(h, P, d_phase, P.blocks[b].phase);
                if (st != QSIM_OK) return st;
                continue;
            }
            TileGeom g;
            FusedMap fm;
            fused_geometry(h->n, k, P.blocks[b].pos, g, fm);
            const uint16_t *bm = reinterpret_cast<const uint16_t *>(d_bmats + per * b);
            CK(launch(h, F_FUSED_TC6, 2.0 * (double)state_bytes(h), 1,
                      [&] { return launch_fused_tc6(h->amp, g, fm, bm, h->d_err, h->sm_count, h->stream); },
                      P.blocks[b].flops),
               "fused block (tensor cores, 6 qubits)");
        }
        return QSIM_OK;
    }
    if (P.tc128) {
        const size_t per = fused_tc128_b_bytes() / sizeof(float);
        for (size_t b = 0; b < P.blocks.size(); b++) {
            // double-float form between the first and the last step of the
            // plan, blocks and phase passes alike
            const bool first = b == 0;
            const bool last = b + 1 == P.blocks.size();
            if (P.blocks[b].phase >= 0) {
                const qsim_status st = run_phase(h, P, d_phase, P.blocks[b].phase, first, last);
                if (st != QSIM_OK) return st;
                continue;
            }
            TileGeom g;
            FusedMap fm;
            fused_geometry(h->n, k, P.blocks[b].pos, g, fm);
            const uint16_t *bm = reinterpret_cast<const uint16_t *>(d_bmats + per * b);
            CK(launch(h, F_FUSED_TC128, 2.0 * (double)state_bytes(h), 1,
                      [&] {
                          return launch_fused_tc128(h->amp, g, fm, bm, h->d_err, h->sm_count, h->stream, first, last);
                      },
                      P.blocks[b].flops),
               "fused block (tensor cores, complex128)");
        }
        return QSIM_OK;
    }
    const size_t per = 2 * (size_t)(2 << k) * (size_t)(2 << k);
    for (size_t b = 0; b < P.blocks.size(); b++) {
        if (P.blocks[b].phase >= 0) {
            const qsim_status st = run_phase(h, P, d_phase, P.blocks[b].phase);
            if (st != QSIM_OK) return st;
            continue;
        }
        TileGeom g;
        FusedMap fm;
        fused_geometry(h->n, k, P.blocks[b].pos, g, fm);
        CK(launch(h, F_FUSED_TC, 2.0 * (double)state_bytes(h), 1,
                  [&] { return launch_fused_tc(h->amp, k, g, fm, d_bmats + per * b, h->d_err, h->sm_count, h->stream); },
                  P.blocks[b].flops),
           "fused block (tensor cores)");
    }
    return QSIM_OK;
}

static qsim_status run_built(qsim_state *h, const qsim_plan_s &P, const TileOp *d_ops, const TilePhase *d_phases) {
    if (!P.blocks.empty())
        return run_blocks(h, P, P.d_bmats ? P.d_bmats : static_cast<const float *>(h->d_dense),
                          P.d_cmats ? P.d_cmats : h->d_dense,
                          P.d_phase ? P.d_phase
                                    : reinterpret_cast<const uint32_t *>(static_cast<const float *>(h->d_dense) +
                                                                         P.bmats.size()));
    if (P.mode == QSIM_MODE_PERGATE) {
        for (const PGate &g : P.sweeps) {
            qsim_status st = sweep_gate(h, g);
            if (st != QSIM_OK) return st;
        }
        return QSIM_OK;
    }
    return launch_passes(h, P.plan, d_ops, d_phases);
}

qsim_status qsim_run_circuit(qsim_handle h, const qsim_gate *gates, size_t ng, const qsim_opts *opts) {
    CHECK_HANDLE(h);
    qsim_plan_s P;
    qsim_status st = build_plan(h, gates, ng, opts, P);
    if (st != QSIM_OK) return st;
    if (!P.blocks.empty()) {
        // block matrices, then the phase passes' tables (right after them)
        const size_t bytes = P.cuda_core ? P.cmats.size() : P.bmats.size() * sizeof(float);
        const size_t pbytes = P.phase_words.size() * sizeof(uint32_t);
        const void *src = P.cuda_core ? static_cast<const void *>(P.cmats.data()) : static_cast<const void *>(P.bmats.data());
        st = ensure_dense(h, bytes + pbytes);
        if (st != QSIM_OK) return st;
        CK(cudaMemcpyAsync(h->d_dense, src, bytes, cudaMemcpyHostToDevice, h->stream), "upload blocks");
        if (pbytes)
            CK(cudaMemcpyAsync(static_cast<unsigned char *>(h->d_dense) + bytes, P.phase_words.data(), pbytes,
                               cudaMemcpyHostToDevice, h->stream),
               "upload phase tables");
        CK(cudaStreamSynchronize(h->stream), "sync");  // the host copy dies with P
        h->h2d += bytes + pbytes;
        return run_built(h, P, nullptr, nullptr);
    }
    if (P.mode == QSIM_MODE_FUSED && !P.plan.ops.empty()) {
        st = upload_program(h, P.plan);
        if (st != QSIM_OK) return st;
    }
    return run_built(h, P, h->d_ops, h->d_phases);
}

static void plan_release(qsim_plan_s *P) {
    if (!P) return;
    for (qsim_plan_s *c : P->cands) plan_release(c);
    for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
    if (P->d_bmats) cudaFree(P->d_bmats);
    if (P->d_cmats) cudaFree(P->d_cmats);
    if (P->d_phase) cudaFree(P->d_phase);
    if (P->d_ops) cudaFree(P->d_ops);
    if (P->d_phases) cudaFree(P->d_phases);
    delete P;
}

// The device copies of a built plan's tables (tile program, block
// matrices) and its final statistics; P is released on failure.
static qsim_status upload_plan(qsim_state *h, qsim_plan_s *P, qsim_plan_s *&out);

static qsim_status create_one(qsim_state *h, const qsim_gate *gates, size_t ng, const qsim_opts *opts,
                              qsim_plan_s *&out) {
    out = nullptr;
    qsim_plan_s *P = new qsim_plan_s;
    const qsim_status st = build_plan(h, gates, ng, opts, *P);
    if (st != QSIM_OK) {
        plan_release(P);
        return st;
    }
    return upload_plan(h, P, out);
}

static qsim_status upload_plan(qsim_state *h, qsim_plan_s *P, qsim_plan_s *&out) {
    out = nullptr;
    qsim_status st = QSIM_OK;
    if (!P->plan.ops.empty()) {
        cudaError_t e = cudaMalloc(&P->d_ops, P->plan.ops.size() * sizeof(TileOp));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_ops, P->plan.ops.data(), P->plan.ops.size() * sizeof(TileOp), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !P->plan.phases.empty()) {
            e = cudaMalloc(&P->d_phases, P->plan.phases.size() * sizeof(TilePhase));
            if (e == cudaSuccess)
                e = cudaMemcpy(P->d_phases, P->plan.phases.data(), P->plan.phases.size() * sizeof(TilePhase),
                               cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) st = cuda_fail(e, "upload plan");
        else h->h2d += P->plan.ops.size() * sizeof(TileOp) + P->plan.phases.size() * sizeof(TilePhase);
    }
    if (st == QSIM_OK && !P->cmats.empty()) {
        cudaError_t e = cudaMalloc(&P->d_cmats, P->cmats.size());
        if (e == cudaSuccess) e = cudaMemcpy(P->d_cmats, P->cmats.data(), P->cmats.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(e, "upload fused blocks");
        else h->h2d += P->cmats.size();
    }
    if (st == QSIM_OK && !P->phase_words.empty()) {
        cudaError_t e = cudaMalloc(&P->d_phase, P->phase_words.size() * sizeof(uint32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_phase, P->phase_words.data(), P->phase_words.size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(e, "upload phase tables");
        else h->h2d += P->phase_words.size() * sizeof(uint32_t);
    }
    if (st == QSIM_OK && !P->bmats.empty()) {
        cudaError_t e = cudaMalloc(&P->d_bmats, P->bmats.size() * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_bmats, P->bmats.data(), P->bmats.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(e, "upload fused blocks");
        else h->h2d += P->bmats.size() * sizeof(float);
    }
    if (st != QSIM_OK) {
        plan_release(P);
        return st;
    }
    P->stats.mode = P->mode;
    P->stats.fuse_k = P->blocks.empty() ? 0 : P->blocks[0].k;
    P->stats.chosen = -1;
    out = P;
    return QSIM_OK;
}

// the stats of an AUTO plan: those of the chosen candidate (the first one
// while tuning) plus the candidate table
static void auto_stats(qsim_plan_s *P) {
    const int shown = P->chosen >= 0 ? P->chosen : 0;
    qsim_plan_stats s = P->cands[shown]->stats;
    s.candidates = (int32_t)P->cands.size();
    s.chosen = P->chosen;
    for (size_t i = 0; i < P->cands.size() && i < 8; i++) {
        s.cand_tile_bits[i] = P->cands[i]->stats.tile_bits;
        s.cand_fuse_k[i] = P->cands[i]->stats.fuse_k;
        s.cand_ms[i] = P->stats.cand_ms[i];
    }
    P->stats = s;
}

qsim_status qsim_plan_create(qsim_handle h, const qsim_gate *gates, size_t ng, const qsim_opts *opts,
                             qsim_plan *out) {
    CHECK_HANDLE(h);
    if (!out) return fail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!opts || opts->mode != QSIM_MODE_AUTO) {
        qsim_plan_s *P = nullptr;
        qsim_status st = create_one(h, gates, ng, opts, P);
        if (st == QSIM_OK) *out = P;
        return st;
    }
    // candidates: tile sizes (and, for complex64, tensor-core fusion widths)
    std::vector<std::pair<int, int>> tk;  // (tile_bits, fuse_k)
    auto add = [&](int T, int k) {
        if (T > h->n) T = h->n;
        for (auto &x : tk)
            if (x.first == T && x.second == k) return;
        tk.push_back({T, k});
    };
    if (h->dt == QSIM_C128) {
        for (int T : {11, 12, 13}) add(T, 0);
        if (fused_tc128_supported(5, h->n)) add(0, 5);
    } else {
        for (int T : {12, 13}) add(T, 0);
        for (int k : {4, 5})
            if (fused_tc_supported((int)h->dt, k, h->n)) add(0, k);
        if (fused_tc6_supported(h->n)) add(0, 6);
    }
    qsim_plan_s *A = new qsim_plan_s;
    A->n = h->n;
    A->dt = h->dt;
    A->mode = QSIM_MODE_AUTO;
    std::memcpy(A->phys, h->phys, sizeof(A->phys));
    for (auto &x : tk) {
        if (A->cands.size() >= 8) break;
        qsim_opts o = *opts;
        o.mode = QSIM_MODE_FUSED;
        o.tile_bits = x.second ? 0 : x.first;
        o.fuse_k = x.second;
        qsim_plan_s *c = nullptr;
        qsim_status st = create_one(h, gates, ng, &o, c);
        // skipped: no tile geometry for a fused width, or a gate wider than it
        // (the tile candidates, planned first, have validated every gate)
        if (st == QSIM_EUNSUPPORTED || (st == QSIM_EINVAL && x.second > 0)) continue;
        if (st != QSIM_OK) {
            plan_release(A);
            return st;
        }
        A->cands.push_back(c);
    }
    if (A->cands.empty()) {
        plan_release(A);
        return fail(QSIM_EUNSUPPORTED, "no candidate plan");
    }
    for (size_t i = 0; i < 2 * A->cands.size(); i++) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            plan_release(A);
            return fail(QSIM_ECUDA, "event");
        }
        A->ev.push_back(e);
    }
    if (A->cands.size() == 1) A->chosen = 0;
    auto_stats(A);
    *out = A;
    return QSIM_OK;
}

static qsim_status run_one(qsim_state *h, qsim_plan_s *p) {
    if (p->n != h->n || p->dt != h->dt || std::memcmp(p->phys, h->phys, sizeof(int) * h->n) != 0)
        return fail(QSIM_EINVAL, "plan was made for another size, dtype or qubit layout");
    return run_built(h, *p, p->d_ops, p->d_phases);
}

qsim_status qsim_plan_run(qsim_handle h, qsim_plan p) {
    CHECK_HANDLE(h);
    if (!p) return fail(QSIM_EINVAL, "null plan");
    if (p->cands.empty()) return run_one(h, p);
    const int nc = (int)p->cands.size();
    if (p->chosen < 0 && p->next >= nc) {
        // every candidate has run once: take the fastest
        int best = 0;
        for (int i = 0; i < nc; i++) {
            float ms = 0.f;
            CK(cudaEventSynchronize(p->ev[2 * i + 1]), "autotune wait");
            CK(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]), "autotune time");
            p->stats.cand_ms[i] = ms;
            if (ms < p->stats.cand_ms[best]) best = i;
        }
        p->chosen = best;
        auto_stats(p);
    }
    if (p->chosen >= 0) return run_one(h, p->cands[p->chosen]);
    const int i = p->next++;
    CK(cudaEventRecord(p->ev[2 * i], h->stream), "autotune start");
    qsim_status st = run_one(h, p->cands[i]);
    CK(cudaEventRecord(p->ev[2 * i + 1], h->stream), "autotune end");
    return st;
}

qsim_status qsim_plan_get_stats(qsim_plan p, qsim_plan_stats *out) {
    if (!p || !out) return fail(QSIM_EINVAL, "null argument");
    *out = p->stats;
    return QSIM_OK;
}

qsim_status qsim_plan_free(qsim_plan p) {
    if (!p) return QSIM_OK;
    cudaDeviceSynchronize();  // runs in flight may still read the plan's tables
    plan_release(p);
    return QSIM_OK;
}

qsim_status qsim_fuse_blocks(int n, const qsim_gate *gates, size_t ng, int k, int32_t *pos, double *U,
                             size_t max_blocks, size_t *nblocks) {
    if (!nblocks || (ng && !gates)) return fail(QSIM_EINVAL, "null argument");
    if (n < 1 || n > kMaxQubits) return fail(QSIM_EINVAL, "n = %d outside [1, %d]", n, kMaxQubits);
    if (k < 1 || k > 6 || k > n) return fail(QSIM_EINVAL, "k = %d outside [1, min(6, n)]", k);
    int ident[64];
    for (int q = 0; q < 64; q++) ident[q] = q;
    std::vector<PGate> pg(ng);
    std::string msg;
    for (size_t i = 0; i < ng; i++)
        if (!prepare_gate(gates[i], n, ident, pg[i], msg)) return fail(QSIM_EINVAL, "gate %zu: %s", i, msg.c_str());
    std::vector<FusedBlock> blocks;
    if (!plan_fused(pg, n, k, blocks)) return fail(QSIM_EINVAL, "a gate acts on more qubits than k");
    *nblocks = blocks.size();
    const size_t ent = (size_t)1 << (2 * k);
    for (size_t b = 0; b < blocks.size() && b < max_blocks; b++) {
        if (pos)
            for (int j = 0; j < k; j++) pos[b * k + j] = blocks[b].pos[j];
        if (U) std::memcpy(U + 2 * ent * b, blocks[b].U.data(), 16 * ent);
    }
    return QSIM_OK;
}

qsim_status qsim_profile_enable(qsim_handle h, int on) {
    CHECK_HANDLE(h);
    h->prof = on != 0;
    return QSIM_OK;
}

qsim_status qsim_profile_read(qsim_handle h, qsim_kernel_time *out, int max, int *count) {
    CHECK_HANDLE(h);
    if (!count || (max > 0 && !out)) return fail(QSIM_EINVAL, "null output");
    CK(cudaStreamSynchronize(h->stream), "sync");
    qsim_kernel_time agg[F_COUNT];
    std::memset(agg, 0, sizeof agg);
    for (auto &r : h->recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        agg[r.fam].launches++;
        agg[r.fam].total_ms += ms;
        agg[r.fam].alg_bytes += r.bytes;
        agg[r.fam].alg_flops += r.flops;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->recs.clear();
    int c = 0;
    for (int f = 0; f < F_COUNT; f++) {
        if (!agg[f].launches) continue;
        if (c < max) {
            out[c] = agg[f];
            std::snprintf(out[c].name, sizeof out[c].name, "%s", kFamName[f]);
        }
        c++;
    }
    *count = c < max ? c : max;
    return QSIM_OK;
}

qsim_status qsim_get_counters(qsim_handle h, qsim_counters *out) {
    CHECK_HANDLE(h);
    if (!out) return fail(QSIM_EINVAL, "null output");
    out->launches = h->launches;
    out->h2d_bytes = h->h2d;
    out->d2h_bytes = h->d2h;
    return QSIM_OK;
}

qsim_status qsim_apply_fused(qsim_handle h, int k, const int *qubits, const double *U) {
    CHECK_HANDLE(h);
    if (k < 1 || k > 6 || k > h->n) return fail(QSIM_EINVAL, "k = %d outside [1, min(6, n)]", k);
    if (!qubits || !U) return fail(QSIM_EINVAL, "qubits or U is NULL");
    int pos[8];
    uint64_t seen = 0;
    for (int j = 0; j < k; j++) {
        if (qubits[j] < 0 || qubits[j] >= h->n) return fail(QSIM_EINVAL, "qubit %d out of range", qubits[j]);
        if ((seen >> qubits[j]) & 1ull) return fail(QSIM_EINVAL, "qubit %d repeated", qubits[j]);
        seen |= 1ull << qubits[j];
        pos[j] = h->phys[qubits[j]];
    }
    const size_t ent = (size_t)1 << (2 * k);
    for (size_t i = 0; i < 2 * ent; i++)
        if (!std::isfinite(U[i])) return fail(QSIM_EINVAL, "non-finite matrix entry");
    const double flops = 8.0 * (double)(1u << k) * std::ldexp(1.0, h->n);
    TileGeom g;
    FusedMap fm;
    if (h->dt == QSIM_C128 && fused_tc128_supported(k, h->n) && fused_geometry(h->n, k, pos, g, fm)) {
        std::vector<uint16_t> b(fused_tc128_b_bytes() / sizeof(uint16_t));
        if (fused_tc128_prepare_b(U, b.data())) {
            const size_t bytes = fused_tc128_b_bytes();
            qsim_status st = ensure_dense(h, bytes);
            if (st != QSIM_OK) return st;
            CK(cudaMemcpyAsync(h->d_dense, b.data(), bytes, cudaMemcpyHostToDevice, h->stream), "upload U");
            CK(cudaStreamSynchronize(h->stream), "sync");  // b is freed on return
            h->h2d += bytes;
            CK(launch(h, F_FUSED_TC128, 2.0 * (double)state_bytes(h), 1,
                      [&] {
                          return launch_fused_tc128(h->amp, g, fm, static_cast<const uint16_t *>(h->d_dense),
                                                    h->d_err, h->sm_count, h->stream, true, true);
                      },
                      flops),
               "fused gate (tensor cores, complex128)");
            return QSIM_OK;
        }
    }
    if (h->dt == QSIM_C64 && k == 6 && fused_tc6_supported(h->n) && fused_geometry(h->n, k, pos, g, fm)) {
        std::vector<uint16_t> b(fused_tc6_b_bytes() / sizeof(uint16_t));
        fused_tc6_prepare_b(U, b.data());
        const size_t bytes = fused_tc6_b_bytes();
        qsim_status st = ensure_dense(h, bytes);
        if (st != QSIM_OK) return st;
        CK(cudaMemcpyAsync(h->d_dense, b.data(), bytes, cudaMemcpyHostToDevice, h->stream), "upload U");
        CK(cudaStreamSynchronize(h->stream), "sync");  // b is freed on return
        h->h2d += bytes;
        CK(launch(h, F_FUSED_TC6, 2.0 * (double)state_bytes(h), 1,
                  [&] {
                      return launch_fused_tc6(h->amp, g, fm, static_cast<const uint16_t *>(h->d_dense), h->d_err,
                                              h->sm_count, h->stream);
                  },
                  flops),
           "fused gate (tensor cores, 6 qubits)");
        return QSIM_OK;
    }
    if (h->dt == QSIM_C64 && fused_tc_supported((int)h->dt, k, h->n) && fused_geometry(h->n, k, pos, g, fm)) {
        // tensor cores: B operand (3xTF32 head and tail) from U
        std::vector<float> b(2 * (size_t)(2 << k) * (size_t)(2 << k));
        fused_tc_prepare_b(k, U, b.data());
        const size_t bytes = b.size() * sizeof(float);
        qsim_status st = ensure_dense(h, bytes);
        if (st != QSIM_OK) return st;
        CK(cudaMemcpyAsync(h->d_dense, b.data(), bytes, cudaMemcpyHostToDevice, h->stream), "upload U");
        CK(cudaStreamSynchronize(h->stream), "sync");  // b is freed on return
        h->h2d += bytes;
        CK(launch(h, F_FUSED_TC, 2.0 * (double)state_bytes(h), 1,
                  [&] {
                      return launch_fused_tc(h->amp, k, g, fm, static_cast<const float *>(h->d_dense), h->d_err,
                                             h->sm_count, h->stream);
                  },
                  flops),
           "fused gate (tensor cores)");
        return QSIM_OK;
    }
    const size_t bytes = ent * amp_bytes(h->dt);
    qsim_status st = ensure_dense(h, bytes);
    if (st != QSIM_OK) return st;
    if (h->dt == QSIM_C64) {
        std::vector<float> f(2 * ent);
        for (size_t i = 0; i < 2 * ent; i++) f[i] = (float)U[i];
        CK(cudaMemcpyAsync(h->d_dense, f.data(), bytes, cudaMemcpyHostToDevice, h->stream), "upload U");
        CK(cudaStreamSynchronize(h->stream), "sync");
    } else {
        CK(cudaMemcpyAsync(h->d_dense, U, bytes, cudaMemcpyHostToDevice, h->stream), "upload U");
        CK(cudaStreamSynchronize(h->stream), "sync");
    }
    h->h2d += bytes;
    CK(launch(h, F_DENSE, 2.0 * (double)state_bytes(h), 1,
              [&] { return launch_dense(h->amp, (int)h->dt, h->n, k, pos, h->d_dense, h->stream); }, flops),
       "dense gate");
    return QSIM_OK;
}

// ---------------------------------------------------------- interchanges
static qsim_status permute_phys(qsim_state *h, int K, const int *l, const int *hb) {
    if (K == 1) {
        PGate pg{};
        pg.kind = QSIM_GATE_SWAP;
        pg.t0 = l[0];
        pg.t1 = hb[0];
        pg.cmask = 0;
        pg.gc = GC_EXCHANGE;
        return sweep_gate(h, pg);
    }
    // K pairs in one pass: a tile holding all 2K bits, one in-tile permutation.
    int T, L, RB;
    qsim_opts po;
    qsim_default_opts(&po);
    po.tile_bits = permute_tile_bits((int)amp_bytes(h->dt));
    tile_defaults(h, &po, T, L, RB);
    L = T;  // runs as long as the tile allows (L shrinks below for pair bits above it)
    uint64_t need = 0;
    for (int i = 0; i < K; i++) need |= (1ull << l[i]) | (1ull << hb[i]);
    if (h->n <= T) {
        T = h->n;
        L = h->n;
    } else {
        // keep the low run length, make room for the pair bits above it
        int above = 0;
        for (int b = 0; b < 64; b++)
            if (((need >> b) & 1ull) && b >= L) above++;
        while (above > T - L && L > 1) {
            L--;
            above = 0;
            for (int b = 0; b < 64; b++)
                if (((need >> b) & 1ull) && b >= L) above++;
        }
        if (above > T - L || above > 10) {
            // more pair bits than one tile holds: the pairs commute, so
            // exchange them in two groups, one pass each
            if (K < 2) return fail(QSIM_EUNSUPPORTED, "pair does not fit a tile");
            const qsim_status st = permute_phys(h, K / 2, l, hb);
            if (st != QSIM_OK) return st;
            return permute_phys(h, K - K / 2, l + K / 2, hb + K / 2);
        }
    }
    TileGeom g{};
    g.n = h->n;
    g.L = L;
    int j = 0;
    uint64_t hm = 0;
    for (int b = L; b < h->n; b++)
        if ((need >> b) & 1ull) hm |= 1ull << b;
    // pad with low-most unused bits above L so the tile has T bits
    for (int b = L; b < h->n && __builtin_popcountll(hm) < T - L; b++) hm |= 1ull << b;
    for (int b = 0; b < 64; b++)
        if ((hm >> b) & 1ull) g.hb[j++] = b;
    g.H = j;
    auto local = [&](int b) -> int {
        if (b < g.L) return b;
        for (int k = 0; k < g.H; k++)
            if (g.hb[k] == b) return g.L + k;
        return -1;
    };
    if (K <= kMaxPermPairs && g.H <= kPermMaxH && g.L >= 1 && g.L + g.H >= 8) {
        // the interchange kernel: tile in shared memory, elements gathered
        // through the permutation, coalesced stores
        PermPairs pp{};
        pp.K = K;
        for (int i = 0; i < K; i++) {
            pp.lo[i] = (int8_t)local(l[i]);
            pp.hi[i] = (int8_t)local(hb[i]);
        }
        CK(launch(h, F_PERM, 2.0 * (double)state_bytes(h), 1,
                  [&] { return launch_permute(h->amp, (int)amp_bytes(h->dt), g, pp, h->d_err, h->sm_count, h->stream); }),
           "interchange pass");
        return QSIM_OK;
    }
    Plan plan;
    TileOp op{};
    op.kind = TOP_PERM;
    op.nperm = K;
    for (int i = 0; i < K; i++) {
        op.pl[i] = (int8_t)local(l[i]);
        op.ph[i] = (int8_t)local(hb[i]);
    }
    plan.ops.push_back(op);
    PassPlan pp{};
    pp.geom = g;
    pp.op_begin = 0;
    pp.op_count = 1;
    plan.passes.push_back(pp);
    qsim_status st = upload_program(h, plan);
    if (st != QSIM_OK) return st;
    return launch_passes(h, plan, h->d_ops, h->d_phases);
}

static qsim_status check_pairs(const qsim_state *h, int K, const int *a, const int *b) {
    if (K < 1 || 2 * K > h->n || K > 8) return fail(QSIM_EINVAL, "K = %d outside [1, min(8, n/2)]", K);
    if (!a || !b) return fail(QSIM_EINVAL, "NULL qubit list");
    uint64_t seen = 0;
    for (int i = 0; i < K; i++) {
        for (int x : {a[i], b[i]}) {
            if (x < 0 || x >= h->n) return fail(QSIM_EINVAL, "qubit %d out of range", x);
            if ((seen >> x) & 1ull) return fail(QSIM_EINVAL, "qubit %d repeated", x);
            seen |= 1ull << x;
        }
    }
    return QSIM_OK;
}

qsim_status qsim_permute_bits(qsim_handle h, int K, const int *l, const int *hb) {
    CHECK_HANDLE(h);
    qsim_status st = check_pairs(h, K, l, hb);
    if (st != QSIM_OK) return st;
    return permute_phys(h, K, l, hb);
}

qsim_status qsim_swap_qubits(qsim_handle h, int K, const int *a, const int *b) {
    CHECK_HANDLE(h);
    qsim_status st = check_pairs(h, K, a, b);
    if (st != QSIM_OK) return st;
    int l[8] = {0}, hb[8] = {0};  // K <= 8 (check_pairs)
    for (int i = 0; i < K; i++) {
        l[i] = h->phys[a[i]];
        hb[i] = h->phys[b[i]];
    }
    st = permute_phys(h, K, l, hb);
    if (st != QSIM_OK) return st;
    for (int i = 0; i < K; i++) std::swap(h->phys[a[i]], h->phys[b[i]]);
    return QSIM_OK;
}

qsim_status qsim_get_layout(qsim_handle h, int *phys) {
    CHECK_HANDLE(h);
    if (!phys) return fail(QSIM_EINVAL, "NULL output");
    for (int q = 0; q < h->n; q++) phys[q] = h->phys[q];
    return QSIM_OK;
}

// ------------------------------------------------------------ measurement
qsim_status qsim_sync(qsim_handle h) {
    CHECK_HANDLE(h);
    return sync_check(h);
}

qsim_status qsim_norm(qsim_handle h, double *out) {
    CHECK_HANDLE(h);
    if (!out) return fail(QSIM_EINVAL, "NULL output");
    CK(launch(h, F_NORM, (double)state_bytes(h), 2,
              [&] { return launch_norm(h->amp, (int)h->dt, h->n, h->d_scratch, h->d_res, h->stream); }),
       "norm");
    CK(cudaMemcpyAsync(h->h_res, h->d_res, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy norm");
    h->d2h += sizeof(double);
    qsim_status st = sync_check(h);
    if (st != QSIM_OK) return st;
    *out = h->h_res[0];
    return QSIM_OK;
}

qsim_status qsim_qubit_probs(qsim_handle h, double *out) {
    CHECK_HANDLE(h);
    if (!out) return fail(QSIM_EINVAL, "NULL output");
    CK(launch(h, F_BITS, (double)state_bytes(h), h->n >= 10 ? 2 : 1,
              [&] { return launch_bit_probs(h->amp, (int)h->dt, h->n, h->d_scratch, h->d_res, h->stream); }),
       "bit marginals");
    CK(cudaMemcpyAsync(h->h_res, h->d_res, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
       "copy marginals");
    h->d2h += h->n * sizeof(double);
    qsim_status st = sync_check(h);
    if (st != QSIM_OK) return st;
    for (int q = 0; q < h->n; q++) out[q] = h->h_res[h->phys[q]];
    return QSIM_OK;
}

qsim_status qsim_qubit_probs_noalloc(const void *amp, int n, qsim_dtype dt, void *stream, double *dev_out) {
    if (!amp || (reinterpret_cast<uintptr_t>(amp) & 15u))
        return fail(QSIM_EINVAL, "amp must be a non-NULL, 16-byte aligned device pointer");
    if (!dev_out) return fail(QSIM_EINVAL, "dev_out is NULL");
    if (n < 1 || n > kMaxQubits)
        return fail(QSIM_EINVAL, "n = %d outside [1, %d]: the static scratch array holds partial sums for at most "
                                 "%d qubits", n, kMaxQubits, kMaxQubits);
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_EINVAL, "bad dtype %d", (int)dt);
    CK(launch_bit_probs_noalloc(amp, (int)dt, n, dev_out, static_cast<cudaStream_t>(stream)),
       "allocation-free marginals");
    return QSIM_OK;
}

static qsim_status ensure_chunk(qsim_state *h) {
    if (h->d_chunk) return QSIM_OK;
    h->chunk_bytes = 64u << 20;
    CK(cudaMalloc(&h->d_chunk, h->chunk_bytes), "cudaMalloc staging");
    return QSIM_OK;
}

qsim_status qsim_probs(qsim_handle h, double *out, size_t len) {
    CHECK_HANDLE(h);
    const uint64_t D = 1ull << h->n;
    if (!out || len != D) return fail(QSIM_EINVAL, "len must be 2^n = %llu", (unsigned long long)D);
    qsim_status st = ensure_chunk(h);
    if (st != QSIM_OK) return st;
    const bool ident = identity_layout(h);
    const uint64_t per = h->chunk_bytes / sizeof(double);
    for (uint64_t s = 0; s < D; s += per) {
        const uint64_t cnt = std::min(per, D - s);
        CK(launch(h, F_PROBS, (double)cnt * (double)(amp_bytes(h->dt) + sizeof(double)), 1,
                  [&] {
                      return launch_probs_chunk(h->amp, (int)h->dt, h->n, h->phys, ident, s, cnt,
                                                static_cast<double *>(h->d_chunk), h->stream);
                  }),
           "probabilities");
        CK(cudaMemcpyAsync(out + s, h->d_chunk, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "copy probabilities");
        h->d2h += cnt * sizeof(double);
        CK(cudaStreamSynchronize(h->stream), "sync");
    }
    return sync_check(h);
}

qsim_status qsim_get_state(qsim_handle h, void *host_out, size_t bytes) {
    CHECK_HANDLE(h);
    if (!host_out || bytes != state_bytes(h)) return fail(QSIM_EINVAL, "need %zu bytes", state_bytes(h));
    if (identity_layout(h)) {
        CK(cudaMemcpyAsync(host_out, h->amp, bytes, cudaMemcpyDeviceToHost, h->stream), "copy state out");
        h->d2h += bytes;
        return sync_check(h);
    }
    qsim_status st = ensure_chunk(h);
    if (st != QSIM_OK) return st;
    const uint64_t D = 1ull << h->n;
    const size_t ab = amp_bytes(h->dt);
    const uint64_t per = h->chunk_bytes / ab;
    for (uint64_t s = 0; s < D; s += per) {
        const uint64_t cnt = std::min(per, D - s);
        CK(launch(h, F_GATHER, 2.0 * (double)cnt * (double)ab, 1,
                  [&] { return launch_gather_chunk(h->amp, (int)h->dt, h->n, h->phys, s, cnt, h->d_chunk, h->stream); }),
           "gather");
        h->d2h += cnt * ab;
        CK(cudaMemcpyAsync(static_cast<char *>(host_out) + s * ab, h->d_chunk, cnt * ab, cudaMemcpyDeviceToHost,
                           h->stream),
           "copy state out");
        CK(cudaStreamSynchronize(h->stream), "sync");
    }
    return sync_check(h);
}

qsim_status qsim_sample(qsim_handle h, const double *u, size_t ns, uint64_t *out) {
    CHECK_HANDLE(h);
    if (ns == 0) return QSIM_OK;
    if (!u || !out) return fail(QSIM_EINVAL, "NULL buffer");
    for (size_t j = 0; j < ns; j++)
        if (!(u[j] >= 0.0 && u[j] < 1.0)) return fail(QSIM_EINVAL, "u[%zu] outside [0, 1)", j);
    const size_t need = sample_scratch_bytes(h->n) + ns * (sizeof(double) + sizeof(uint64_t)) + 256;
    void *buf = nullptr;
    CK(cudaMallocAsync(&buf, need, h->stream), "cudaMallocAsync sample buffers");
    double *du = static_cast<double *>(buf);
    uint64_t *dout = reinterpret_cast<uint64_t *>(du + ns);
    double *scr = reinterpret_cast<double *>(dout + ns);
    cudaError_t e = cudaMemcpyAsync(du, u, ns * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    h->h2d += ns * sizeof(double);
    h->d2h += ns * sizeof(uint64_t);
    const bool ident = identity_layout(h);
    if (e == cudaSuccess)
        e = launch(h, F_SAMPLE, (double)state_bytes(h) * 2.0, 3, [&] {
            return launch_sample(h->amp, (int)h->dt, h->n, h->phys, ident, du, ns, dout, scr, h->stream);
        });
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, ns * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(buf, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sample");
    return sync_check(h);
}

// ------------------------------------------------------------------ batch
struct qsim_batch_s {
    std::vector<qsim_handle> states;
    std::vector<uint64_t> x0;
    cudaStream_t stream = nullptr;   // where runs are enqueued (cs[0]'s stream)
    cudaStream_t cap = nullptr;      // private stream used for graph capture
    void *dbuf = nullptr;            // circuits, passes, ops, items, counters, done, error word
    BatchCircuit *d_circs = nullptr;
    BatchPass *d_passes = nullptr;
    TileOp *d_ops = nullptr;
    TilePhase *d_phases = nullptr;
    BatchItem *d_items = nullptr;
    uint32_t *d_counters = nullptr;  // 64-bit item counter, then one counter per pass
    uint32_t *d_err = nullptr;
    size_t zero_bytes = 0;           // counters + done + error word, cleared before each run
    uint64_t nitems = 0;
    long long budget = 0;
    int sm_count = 152;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t *h_err = nullptr;       // pinned
    qsim_batch_stats stats{};
    // circuits run as dense blocks on the tensor cores after the persistent
    // launch: their state, basis index and plan
    std::vector<qsim_handle> fused_states;
    std::vector<uint64_t> fused_x0;
    std::vector<qsim_plan_s *> fused_plans;
};

// Circuits of at least this many qubits take the tensor-core lane of a batch
// (they carry almost all of a mixed batch's bytes; below it a block's launch
// costs more than its pass).
constexpr int kBatchFusedMinQubits = 20;

static void batch_release(qsim_batch_s *b) {
    if (!b) return;
    for (qsim_plan_s *P : b->fused_plans) plan_release(P);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dbuf) cudaFree(b->dbuf);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->h_err) cudaFreeHost(b->h_err);
    delete b;
}

static cudaError_t batch_enqueue(qsim_batch_s *b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, b->zero_bytes, s);
    if (e != cudaSuccess) return e;
    if (b->nitems) {
        e = launch_batch(b->d_circs, b->d_passes, b->d_ops, b->d_phases, b->d_items, b->nitems, b->d_counters,
                         b->d_counters + 2, b->d_err, b->budget, b->sm_count, s);
        if (e != cudaSuccess) return e;
    }
    // the tensor-core lane: |x0> and the blocks of every such circuit, on the
    // same stream, with the batch's error word (so a timeout there is
    // reported like one in the persistent launch)
    for (size_t i = 0; i < b->fused_plans.size(); i++) {
        qsim_state *h = b->fused_states[i];
        const cudaStream_t hs = h->stream;
        uint32_t *const herr = h->d_err;
        const bool prof = h->prof;
        h->stream = s;
        h->d_err = b->d_err;
        h->prof = false;
        e = launch_init_basis(h->amp, (int)h->dt, h->n, b->fused_x0[i], s);
        if (e == cudaSuccess && run_built(h, *b->fused_plans[i], nullptr, nullptr) != QSIM_OK) e = cudaErrorUnknown;
        h->stream = hs;
        h->d_err = herr;
        h->prof = prof;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// capture: record the runs' launches in a CUDA graph (a planned batch replays
// it; a one-shot batch enqueues its launches directly).
static qsim_status batch_create(const qsim_circuit *cs, size_t nc, const qsim_opts *opts, qsim_batch *out,
                                bool capture) {
    if (!out) return fail(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (nc == 0 || !cs) return fail(QSIM_EINVAL, "empty batch");
    qsim_opts o;
    qsim_default_opts(&o);
    if (opts) o = *opts;
    int dev = -1;
    for (size_t i = 0; i < nc; i++) {
        const qsim_handle h = cs[i].state;
        if (!h) return fail(QSIM_EINVAL, "circuit %zu has no state", i);
        if (h->dt != QSIM_C64) return fail(QSIM_EINVAL, "batch states must be complex64");
        if (h->n > 24) return fail(QSIM_EINVAL, "batch states have at most 24 qubits");
        if (dev < 0) dev = h->device;
        if (h->device != dev) return fail(QSIM_EINVAL, "batch states must share one device");
        if (h->n < 64 && cs[i].x0 >= (1ull << h->n)) return fail(QSIM_EINVAL, "circuit %zu: x0 out of range", i);
        if (cs[i].ng && !cs[i].gates) return fail(QSIM_EINVAL, "circuit %zu: gates is NULL", i);
    }
    const int Tmax = (o.tile_bits > 0 && o.tile_bits < 12) ? o.tile_bits : 12;
    std::vector<BatchCircuit> circs(nc);
    std::vector<BatchPass> passes;
    std::vector<TileOp> ops;
    std::vector<TilePhase> phases;
    std::vector<std::vector<int>> pass_of(nc);
    int max_passes = 0;
    int64_t ngates = 0;
    double alg_bytes = 0.0, alg_flops = 0.0;
    int ident[64];
    for (int q = 0; q < 64; q++) ident[q] = q;
    std::vector<qsim_plan_s *> fplans(nc, nullptr), built(nc, nullptr);  // uploaded / planned on the host only
    auto free_fplans = [&]() {
        for (qsim_plan_s *P : fplans) plan_release(P);
        for (qsim_plan_s *P : built) plan_release(P);
    };
    // The tensor-core lane: 6-qubit blocks (or fuse_k) for the largest
    // circuits, unless fuse_k = -1.  Their FP64 block products are planned on
    // the host in parallel threads (the planner is pure host code); a circuit
    // with a gate wider than the block stays in the persistent launch.
    const int fk = o.fuse_k > 0 ? o.fuse_k : 6;
    std::vector<size_t> lane;
    for (size_t i = 0; i < nc; i++) {
        const qsim_handle h = cs[i].state;
        if (o.fuse_k >= 0 && h->n >= kBatchFusedMinQubits && cs[i].ng > 0 &&
            ((fk == 6 && fused_tc6_supported(h->n)) || (fk != 6 && fused_tc_supported(0, fk, h->n)))) {
            for (int q = 0; q < 64; q++) h->phys[q] = q;  // every run starts from the identity layout
            lane.push_back(i);
        }
    }
    std::vector<qsim_status> built_st(nc, QSIM_OK);
    {
        qsim_opts fo = o;
        fo.mode = QSIM_MODE_FUSED;
        fo.tile_bits = 0;
        fo.fuse_k = fk;
        std::atomic<size_t> next{0};
        auto work = [&]() {
            for (size_t j = next++; j < lane.size(); j = next++) {
                const size_t i = lane[j];
                qsim_plan_s *P = new qsim_plan_s;
                built_st[i] = build_plan(cs[i].state, cs[i].gates, cs[i].ng, &fo, *P, false);
                if (built_st[i] == QSIM_OK) built[i] = P;
                else plan_release(P);
            }
        };
        const size_t nthr = std::min<size_t>(lane.size(), std::max(1u, std::min(32u, std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        for (size_t t = 1; t < nthr; t++) pool.emplace_back(work);
        work();
        for (std::thread &t : pool) t.join();
    }
    int64_t nfused = 0;
    for (size_t i = 0; i < nc; i++) {
        const qsim_handle h = cs[i].state;
        if (built[i] || built_st[i] != QSIM_OK) {
            qsim_plan_s *P = nullptr;
            qsim_status fst = built_st[i];
            if (built[i]) fst = upload_plan(h, built[i], P);
            built[i] = nullptr;
            if (fst == QSIM_OK) {
                fplans[i] = P;
                ngates += (int64_t)cs[i].ng;
                alg_bytes += P->stats.alg_bytes;
                alg_flops += P->stats.alg_flops;
                circs[i].amp = h->amp;
                circs[i].x0 = cs[i].x0;
                circs[i].pass_begin = (int32_t)passes.size();
                circs[i].npasses = 0;  // no items in the persistent launch
                nfused++;
                continue;
            }
            if (fst != QSIM_EINVAL && fst != QSIM_EUNSUPPORTED) {
                free_fplans();
                return fail(fst, "circuit %zu: planning its dense blocks failed", i);
            }
        }
        std::vector<PGate> pg(cs[i].ng);
        std::string msg;
        for (size_t k = 0; k < cs[i].ng; k++)
            if (!prepare_gate(cs[i].gates[k], h->n, ident, pg[k], msg)) {
                free_fplans();
                return fail(QSIM_EINVAL, "circuit %zu gate %zu: %s", i, k, msg.c_str());
            }
        ngates += (int64_t)cs[i].ng;
        const int T = h->n < Tmax ? h->n : Tmax;
        const int L = T < 5 ? T : 5;
        Plan plan;
        // 12-bit tiles of complex64 circuits run the register program
        const int RB = (T == 12 && tile2_supported(0, T)) ? kBatchRB : 0;
        plan_tiles(pg, h->n, T, L, plan, RB, kRegMaxOps, kRegMaxPhases);  // k_batch stages every pass
        circs[i].amp = h->amp;
        circs[i].x0 = cs[i].x0;
        circs[i].pass_begin = (int32_t)passes.size();
        if (plan.passes.empty()) {  // no gates: one pass that only writes |x0>
            PassPlan pp{};
            pp.geom.n = h->n;
            pp.geom.L = T < 5 ? T : 5;
            pp.geom.H = T - pp.geom.L;
            for (int k = 0; k < pp.geom.H; k++) pp.geom.hb[k] = pp.geom.L + k;
            plan.passes.push_back(pp);
        }
        for (const PassPlan &pp : plan.passes) {
            if (pp.op_count > kRegMaxOps || pp.phase_count > kRegMaxPhases) {  // the planner's cap guarantees this
                free_fplans();
                return fail(QSIM_EUNSUPPORTED, "circuit %zu: a pass exceeds the staged program capacity", i);
            }
            alg_bytes += 2.0 * (double)state_bytes(h);  // each pass reads and writes the state once
            alg_flops += pp.flops;
            BatchPass bp{};
            bp.geom = pp.geom;
            bp.op_begin = (int32_t)ops.size();
            bp.op_count = pp.op_count;
            bp.ntiles = 1u << (h->n - (pp.geom.L + pp.geom.H));
            bp.phase_begin = (int32_t)phases.size();
            bp.phase_count = pp.phase_count;
            for (int k = 0; k < pp.phase_count; k++) {  // op indices rebased into the batch's op array
                TilePhase ph = plan.phases[pp.phase_begin + k];
                ph.op_begin = ph.op_begin - pp.op_begin + bp.op_begin;
                phases.push_back(ph);
            }
            ops.insert(ops.end(), plan.ops.begin() + pp.op_begin, plan.ops.begin() + pp.op_begin + pp.op_count);
            passes.push_back(bp);
        }
        circs[i].npasses = (int32_t)plan.passes.size();
        max_passes = std::max(max_passes, circs[i].npasses);
    }
    std::vector<BatchItem> items;
    for (int p = 0; p < max_passes; p++)
        for (size_t i = 0; i < nc; i++) {
            if (p >= circs[i].npasses) continue;
            const uint32_t nt = passes[circs[i].pass_begin + p].ntiles;
            for (uint32_t t = 0; t < nt; t++) items.push_back(BatchItem{(uint32_t)i, (uint32_t)p, t});
        }
    qsim_batch_s *b = new qsim_batch_s;
    for (size_t i = 0; i < nc; i++) {
        b->states.push_back(cs[i].state);
        b->x0.push_back(cs[i].x0);
        if (fplans[i]) {
            b->fused_states.push_back(cs[i].state);
            b->fused_x0.push_back(cs[i].x0);
            b->fused_plans.push_back(fplans[i]);  // owned by the batch from here on
        }
    }
    b->stream = cs[0].state->stream;
    b->sm_count = cs[0].state->sm_count;
    b->nitems = items.size();
    b->budget = (o.wait_budget_us > 0 ? (long long)o.wait_budget_us : 2000000ll) * 2000ll;  // ~2 GHz SM clock
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t sc = al(circs.size() * sizeof(BatchCircuit)), sp = al(passes.size() * sizeof(BatchPass));
    const size_t so = al(std::max<size_t>(ops.size(), 1) * sizeof(TileOp)), si = al(items.size() * sizeof(BatchItem));
    const size_t sh = al(std::max<size_t>(phases.size(), 1) * sizeof(TilePhase));
    b->zero_bytes = 8 + passes.size() * 4 + 4 + 4;
    const size_t sz = al(b->zero_bytes);
    cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaMalloc(&b->dbuf, sc + sp + so + si + sz + sh);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_err, sizeof(uint32_t));
    if (e != cudaSuccess) {
        batch_release(b);
        return cuda_fail(e, "batch buffers");
    }
    char *base = static_cast<char *>(b->dbuf);
    b->d_circs = reinterpret_cast<BatchCircuit *>(base);
    b->d_passes = reinterpret_cast<BatchPass *>(base + sc);
    b->d_ops = reinterpret_cast<TileOp *>(base + sc + sp);
    b->d_items = reinterpret_cast<BatchItem *>(base + sc + sp + so);
    b->d_counters = reinterpret_cast<uint32_t *>(base + sc + sp + so + si);
    b->d_err = b->d_counters + 2 + passes.size();
    b->d_phases = reinterpret_cast<TilePhase *>(base + sc + sp + so + si + sz);
    e = cudaMemcpy(b->d_circs, circs.data(), circs.size() * sizeof(BatchCircuit), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_passes, passes.data(), passes.size() * sizeof(BatchPass), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ops.empty())
        e = cudaMemcpy(b->d_ops, ops.data(), ops.size() * sizeof(TileOp), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !phases.empty())
        e = cudaMemcpy(b->d_phases, phases.data(), phases.size() * sizeof(TilePhase), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        batch_release(b);
        return cuda_fail(e, "batch upload");
    }
    // capture: counter reset, the persistent launch and the tensor-core lane,
    // replayed by every run
    if (capture && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaError_t le = batch_enqueue(b, b->cap);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
        if (le == cudaSuccess && ce == cudaSuccess && g &&
            cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
            b->graph = g;
        } else {
            if (g) cudaGraphDestroy(g);
            b->exec = nullptr;
        }
    }
    cudaGetLastError();  // a refused capture leaves no sticky error: fall back to direct launches
    b->stats.circuits = (int64_t)nc;
    b->stats.gates = ngates;
    int64_t nblocks = 0;
    for (qsim_plan_s *P : b->fused_plans) nblocks += (int64_t)P->blocks.size();
    b->stats.passes = (int64_t)passes.size();
    b->stats.blocks = nblocks;
    b->stats.items = (int64_t)items.size();
    b->stats.fused = (int32_t)nfused;
    b->stats.kernels = (items.empty() ? 0 : 1) + nfused + nblocks;  // persistent launch, |x0> and blocks
    b->stats.alg_bytes = alg_bytes;
    b->stats.alg_flops = alg_flops;
    b->stats.graph = b->exec ? 1 : 0;
    *out = b;
    return QSIM_OK;
}

qsim_status qsim_batch_create(const qsim_circuit *cs, size_t nc, const qsim_opts *opts, qsim_batch *out) {
    return batch_create(cs, nc, opts, out, true);
}

qsim_status qsim_batch_run(qsim_batch b) {
    if (!b) return fail(QSIM_EINVAL, "null batch");
    for (qsim_handle h : b->states)
        for (int q = 0; q < 64; q++) h->phys[q] = q;
    if (b->exec) {
        CK(cudaGraphLaunch(b->exec, b->stream), "batch graph launch");
    } else {
        CK(batch_enqueue(b, b->stream), "batch launch");
    }
    for (qsim_handle h : b->states) h->launches += 1;
    return QSIM_OK;
}

qsim_status qsim_batch_sync(qsim_batch b) {
    if (!b) return fail(QSIM_EINVAL, "null batch");
    CK(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream), "read error word");
    CK(cudaStreamSynchronize(b->stream), "sync");
    if (*b->h_err) return fail(QSIM_ETIMEOUT, "a bounded wait between batch passes expired");
    return QSIM_OK;
}

qsim_status qsim_batch_get_stats(qsim_batch b, qsim_batch_stats *out) {
    if (!b || !out) return fail(QSIM_EINVAL, "null argument");
    *out = b->stats;
    return QSIM_OK;
}

qsim_status qsim_batch_free(qsim_batch b) {
    if (!b) return QSIM_OK;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    return QSIM_OK;
}

qsim_status qsim_run_batch(const qsim_circuit *cs, size_t nc, const qsim_opts *opts) {
    if (nc == 0) return QSIM_OK;
    qsim_batch b = nullptr;
    qsim_status st = batch_create(cs, nc, opts, &b, false);  // one run: no graph to build
    if (st != QSIM_OK) return st;
    st = qsim_batch_run(b);
    if (st == QSIM_OK) st = qsim_batch_sync(b);
    qsim_batch_free(b);
    return st;
}

}  // extern "C"
