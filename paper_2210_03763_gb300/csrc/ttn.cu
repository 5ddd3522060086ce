// libttn host side: tree, environments, TDVP sweep and the C ABI (include/ttn.h).
//
// Method (Sec. "Tensor network simulations"): binary TTN over the
// Hilbert-curve leaf order, single-site TDVP.  One step of dt is a forward
// half-sweep with tau = dt/2 (post-order: for each child node, gauge move
// down, recurse, QR back up and evolve the link backwards; then evolve the
// node forwards) followed by its exact reverse.  H is frozen at t + dt/2.
//
// Every contraction is one launch of the strided complex GEMM (GemmArgs);
// Lanczos, QR and the small tridiagonal exponential are in kernels.cu and
// qr.cu.  All state lives on the device; the host only orders launches and
// reads the Krylov convergence flag once per Lanczos step.
#include "common.cuh"
#include "../../include/ttn.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

namespace {

typedef std::complex<double> zc;
constexpr int MAX_CHI = 256;
constexpr int MAX_ATOMS = 1024;

struct TtnError : std::runtime_error {
    ttn_status code;
    TtnError(ttn_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CUDA_OK(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw TtnError(TTN_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

inline cplx C(double re, double im = 0.0) { return make_double2(re, im); }

// ------------------------------------------------------------------ tree
struct Node {
    int child[2];        // >= 0 node id, else -(leaf + 1)
    int parent = -1;
    int level = 0;
    int d[3];
    long long s = 0;
    std::vector<int> sites;   // real atoms in the subtree, leaf order
};

// Hilbert curve on a side x side grid: cell visited at step d (own copy of
// the iterative index -> (x, y) map, starting at the (0, 0) corner).
void hilbert_cell(int side, int d, int& x, int& y) {
    x = y = 0;
    int t = d;
    for (int s = 1; s < side; s *= 2) {
        int rx = 1 & (t / 2);
        int ry = 1 & (t ^ rx);
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - x;
                y = s - 1 - y;
            }
            std::swap(x, y);
        }
        x += s * rx;
        y += s * ry;
        t /= 4;
    }
}

// ------------------------------------------------------------ environments
// Environment of the atoms S behind one leg, in that leg's basis (dim D):
// H = static block Hamiltonian (all n_i n_j terms inside S), n_i for every
// atom of S, and (sx, sz, |r><1|) for the driven atoms of S.
struct Env {
    int D = 1;
    std::vector<int> sites;
    std::vector<int> driven;
    bool has_H = false;            // false: static block is zero
    cplx* H = nullptr;             // D*D
    cplx* nops = nullptr;          // |sites| * D*D
    cplx* dops = nullptr;          // 3 * |driven| * D*D
    int* d_sites = nullptr;        // device copies of the id lists
    int* d_driven = nullptr;
    size_t cap_n = 0, cap_d = 0;   // capacity in matrices
};

struct Pair {  // channel side a (r = |S_a| channels), G side b
    int a, b;
    int r;
    const cplx* Na;     // n ops of env a (r matrices of D_a^2)
    cplx* G;            // r matrices of D_b^2 (filled per visit)
};

}  // namespace

struct ttn_ctx {
    int Lx = 0, Ly = 0, N = 0, chi = 0;
    int n_leaves = 0;
    std::vector<int> leaf_atom;
    std::vector<Node> nodes;
    int root = 0;
    std::vector<std::vector<int>> level_nodes;
    cudaStream_t stream = nullptr;
    ttn_precision prec = TTN_FP64;
    std::string err;
    double t = 0.0;
    int centre = -1;

    std::vector<double> xy;
    double C6 = 0.0, r_cut = 0.0;
    double gamma = 0.0;                    // decay rate of Eq. 3 (0: closed system)
    std::vector<double> V;                 // N x N
    std::vector<ttn_pulse> schedule;
    std::vector<int> driven;               // per atom
    double* d_coef = nullptr;              // 5 * N
    std::vector<double> h_coef;

    // device tensors: one buffer per node plus scratch, all of capacity smax
    long long smax = 0;
    std::vector<cplx*> T;
    cplx* tmp[3] = {nullptr, nullptr, nullptr};
    cplx* Z = nullptr;        // channel / op stack scratch
    long long zcap = 0;       // capacity in complex
    cplx* Gbuf[3] = {nullptr, nullptr, nullptr};
    long long gcap = 0;
    cplx* hb[3] = {nullptr, nullptr, nullptr};
    cplx* Rbuf = nullptr;
    cplx* dense_H = nullptr;  // SMALL_S^2: dense H_eff of a small node or link
    cplx* Kbasis = nullptr;   // (KRYLOV_MMAX + 1) * smax
    KrylovScalars* ks = nullptr;
    cplx* kh1 = nullptr;      // KRYLOV_MMAX + 1
    cplx* kh2 = nullptr;
    cplx* kpart = nullptr;    // 2 * RED_BLOCKS * (KRYLOV_MMAX + 1)
    double* kpn = nullptr;    // RED_BLOCKS
    double* apx = nullptr;    // RED_BLOCKS: norm^2 partials of an absorbed node
    double* apr = nullptr;    // RED_BLOCKS: norm^2 partials of the absorbed link matrix
    int* hflag = nullptr;     // pinned host: converged, nonfinite
    QrScratch qr{};
    std::map<std::pair<int, int>, int*> cand;   // (node, leg) -> candidate rows
    std::map<std::pair<int, int>, int> ncand;

    std::vector<Env> up, down, phys;
    Env dummy;
    std::map<std::pair<const Env*, const Env*>, std::pair<double*, cplx*>> vsub;   // G-stack weights

    // kernel-level profile: event pairs around launches while enabled
    bool profiling = false;
    struct ProfRec { int kind; cudaEvent_t e0, e1; double flops, bytes; int shape[4]; };
    std::vector<std::array<double, 7>> prof_last;   // kind, M, N, K, batch, ms, flops of the last profile
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    void* split_ws = nullptr;   // packed operands of the split GEMM (+ error flag)
    size_t split_cap = 0;
    void* f64_ws = nullptr;     // split-K partial sums of FP64 contractions
    size_t f64_cap = 0;
    // split-precision H_eff of one node visit (see SplitHeff): per leg the
    // stacked operand planes [X | channel stacks] and the operator stack,
    // per channel pair the packed G stack; grown on demand, zeroed when
    // allocated so that every float the MMAs can read is finite
    float* shP[3] = {nullptr, nullptr, nullptr};
    size_t shP_cap[3] = {0, 0, 0};
    float* shQ[3] = {nullptr, nullptr, nullptr};
    size_t shQ_cap[3] = {0, 0, 0};
    float* shG[3] = {nullptr, nullptr, nullptr};
    size_t shG_cap[3] = {0, 0, 0};
    float* shX[3] = {nullptr, nullptr, nullptr};
    size_t shX_cap[3] = {0, 0, 0};
    int64_t stats[6] = {0, 0, 0, 0, 0, 0};
    double max_err = 0.0;
    std::vector<void*> allocs;
};

// ---- test hooks (ttn_test_inject): host-side fault injection ----------------
static std::atomic<long long> g_inj_tc_stall{0};     // tensor-core launches still to stall
static std::atomic<int> g_inj_mmax{0};               // Krylov dimension cap, 0: KRYLOV_MMAX
static std::atomic<long long> g_inj_alloc_fail{0};   // device allocations still to fail
constexpr unsigned long long INJ_STALL_NS = 1000000ull;   // 1 ms wait that runs out

namespace {

// Take one unit from a pending-count hook (false when none is pending).
bool take_one(std::atomic<long long>& n) {
    long long v = n.load();
    while (v > 0)
        if (n.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

}  // namespace

unsigned long long test_take_tc_stall() { return take_one(g_inj_tc_stall) ? INJ_STALL_NS : 0ull; }
int test_krylov_mmax() {
    const int m = g_inj_mmax.load();
    return (m >= 1 && m < KRYLOV_MMAX) ? m : KRYLOV_MMAX;
}
bool test_take_alloc_fail() { return take_one(g_inj_alloc_fail); }

namespace {

void* dalloc(ttn_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (test_take_alloc_fail()) throw TtnError(TTN_ERR_ALLOC, "cudaMalloc: injected failure");
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) throw TtnError(TTN_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->allocs.push_back(p);
    return p;
}

long long ipow3_capped(int k, long long cap) {
    long long v = 1;
    for (int i = 0; i < k; ++i) {
        v *= 3;
        if (v >= cap) return cap;
    }
    return v;
}

int leg_dim(const ttn_ctx* c, int k, int leg) { return c->nodes[k].d[leg]; }

// ------------------------------------------------------------------ GEMMs
void grow_split_ws(ttn_ctx* c, size_t bytes) {
    if (bytes <= c->split_cap) return;
    CUDA_OK(cudaStreamSynchronize(c->stream));
    int flag = 0;
    if (c->split_ws) {
        CUDA_OK(cudaMemcpy(&flag, c->split_ws, sizeof(int), cudaMemcpyDeviceToHost));
        cudaFree(c->split_ws);
        c->split_ws = nullptr;
        c->split_cap = 0;
    }
    size_t cap = bytes + bytes / 4;
    if (test_take_alloc_fail() || cudaMalloc(&c->split_ws, cap) != cudaSuccess)
        throw TtnError(TTN_ERR_ALLOC, "split workspace");
    CUDA_OK(cudaMemcpy(c->split_ws, &flag, sizeof(int), cudaMemcpyHostToDevice));
    c->split_cap = cap;
}

// Profile kinds: 0 tensor-core GEMM, 1 split packing, 2 FP64 GEMM, 3 QR,
// 4 Krylov vector work (re-orthogonalisation, scalars, combination, and the
// one-block Krylov runs of small nodes), 5 the remaining element-wise
// kernels of the sweep (block assembly, leg permutations, absorb norms).
enum { PK_TC = 0, PK_PACK = 1, PK_F64 = 2, PK_QR = 3, PK_KRY = 4, PK_MISC = 5, PK_N = 6 };

cudaEvent_t next_event(ttn_ctx* c) {
    if (c->ev_next == c->ev_pool.size()) {
        cudaEvent_t e;
        CUDA_OK(cudaEventCreate(&e));
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_next++];
}

struct ProfScope {
    ttn_ctx* c;
    int kind;
    double flops, bytes;
    int shape[4] = {0, 0, 0, 0};
    cudaEvent_t e0 = nullptr;
    ProfScope(ttn_ctx* c_, int k, double f = 0, double b = 0, const GemmArgs* g = nullptr)
        : c(c_), kind(k), flops(f), bytes(b) {
        if (g) {
            shape[0] = g->M;
            shape[1] = g->N;
            shape[2] = g->Ki * g->Ko;
            shape[3] = g->Bi * g->Bo;
        }
        if (c->profiling) {
            e0 = next_event(c);
            CUDA_OK(cudaEventRecord(e0, c->stream));
        }
    }
    ~ProfScope() {
        if (c->profiling && e0) {
            cudaEvent_t e1 = next_event(c);
            cudaEventRecord(e1, c->stream);
            c->prof.push_back({kind, e0, e1, flops, bytes, {shape[0], shape[1], shape[2], shape[3]}});
        }
    }
};

double gemm_flops(const GemmArgs& g) {
    return 8.0 * g.M * (double)g.N * g.Ki * (double)g.Ko * g.Bi * (double)g.Bo;
}

// Observables and gauge-only moves always run in FP64 (ForceFp64): the
// tensor core's FP32 accumulation rounds with a small bias (results shrink by
// ~1e-7 relative), which in a contraction that writes the state is a norm
// loss, while in an H_eff product or an environment it only perturbs the
// generator (the Lanczos propagator stays unitary).  The sweep's own link
// absorbs run in split precision with an exact FP64 norm restore (absorb).
thread_local bool g_force_fp64 = false;
struct ForceFp64 {
    bool old;
    ForceFp64() : old(g_force_fp64) { g_force_fp64 = true; }
    ~ForceFp64() { g_force_fp64 = old; }
};

void gemm(ttn_ctx* c, const GemmArgs& g) {
    int n = -1;
    const double fl = gemm_flops(g);
    if (c->prec == TTN_SPLIT_TF32X3 && !g_force_fp64) {
        size_t need = split_workspace_bytes(g);
        if (need > 0) {
            grow_split_ws(c, need);
            double nb = (double)g.Bi * g.Bo;
            double pack_bytes = nb * ((double)g.M + g.N) * g.Ki * (double)g.Ko * 16.0 + 0.5 * need;
            {
                ProfScope ps(c, PK_PACK, 0.0, pack_bytes, &g);
                n = launch_split_pack(g, c->stream, c->split_ws, c->split_cap);
            }
            if (n >= 0) {
                ProfScope ps(c, PK_TC, fl, 0.5 * need + nb * (double)g.M * g.N * 16.0, &g);
                int m = launch_split_mma(g, c->stream, c->split_ws, c->split_cap);
                if (m < 0) throw TtnError(TTN_ERR_CUDA, "split GEMM launch failed after packing");
                n += m;
            }
        }
    }
    if (n < 0) {
        const size_t wb = f64_workspace_bytes(g);
        if (wb > c->f64_cap) {   // split-K partials of small-output FP64 contractions
            CUDA_OK(cudaStreamSynchronize(c->stream));
            if (c->f64_ws) cudaFree(c->f64_ws);
            c->f64_ws = nullptr;
            c->f64_cap = 0;
            const size_t want = wb + wb / 4;
            if (test_take_alloc_fail() || cudaMalloc(&c->f64_ws, want) != cudaSuccess) {
                c->f64_ws = nullptr;
                throw TtnError(TTN_ERR_ALLOC, "FP64 split-K workspace");
            }
            c->f64_cap = want;
        }
        ProfScope ps(c, PK_F64, fl, 0.0, &g);
        n = launch_zgemm_f64(g, c->stream, c->f64_ws, c->f64_cap);
    }
    c->stats[3] += n;
}

// A bounded device-side wait of the split GEMM gave up -> TTN_ERR_TIMEOUT.
void check_split_flag(ttn_ctx* c) {
    if (!c->split_ws) return;
    int flag = 0;
    CUDA_OK(cudaMemcpyAsync(&flag, c->split_ws, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    if (flag) {   // clear it so that the context can be used again once its state is reloaded
        const int zero = 0;
        CUDA_OK(cudaMemcpy(c->split_ws, &zero, sizeof(int), cudaMemcpyHostToDevice));
        throw TtnError(TTN_ERR_TIMEOUT, "tensor-core GEMM pipeline wait timed out");
    }
}

GemmArgs base_args() {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.Ki = g.Ko = g.Bi = g.Bo = 1;
    g.alpha = C(1.0);
    g.beta = C(0.0);
    return g;
}

// Y = alpha * M x_leg X + beta * Y for nb stacked matrices M (stride m_bs) and
// outputs (stride y_bs).  M is Dout x Din column-major; X has dims d with
// d[leg] = Din; Y has dims d with d[leg] = Dout.
void leg_apply(ttn_ctx* c, const cplx* M, int Dout, const cplx* X, const int* d, int leg, cplx* Y,
               double beta, int nb = 1, long long m_bs = 0, long long y_bs = 0, bool conjM = false) {
    GemmArgs g = base_args();
    g.beta = C(beta);
    int d0 = d[0], d1 = d[1], d2 = d[2];
    int Din = d[leg];
    g.conjA = g.conjB = 0;
    if (leg == 0) {
        g.M = Dout; g.N = d1 * d2; g.Ki = Din;
        g.A = M; g.a_m = 1; g.a_ki = Dout; g.conjA = conjM;
        g.B = X; g.b_ki = 1; g.b_n = d0;
        g.C = Y; g.c_m = 1; g.c_n = Dout;
        g.Bi = nb; g.a_bi = m_bs; g.b_bi = 0; g.c_bi = y_bs;
    } else if (leg == 1) {
        g.M = d0; g.N = Dout; g.Ki = Din;
        g.A = X; g.a_m = 1; g.a_ki = d0; g.a_bi = (long long)d0 * d1;
        g.B = M; g.b_ki = Dout; g.b_n = 1; g.conjB = conjM;
        g.C = Y; g.c_m = 1; g.c_n = d0; g.c_bi = (long long)d0 * Dout;
        g.Bi = d2;
        g.Bo = nb; g.a_bo = 0; g.b_bo = m_bs; g.c_bo = y_bs;
    } else {
        g.M = d0 * d1; g.N = Dout; g.Ki = Din;
        g.A = X; g.a_m = 1; g.a_ki = (long long)d0 * d1;
        g.B = M; g.b_ki = Dout; g.b_n = 1; g.conjB = conjM;
        g.C = Y; g.c_m = 1; g.c_n = (long long)d0 * d1;
        g.Bi = nb; g.a_bi = 0; g.b_bi = m_bs; g.c_bi = y_bs;
    }
    gemm(c, g);
}

// Y += sum_i N_i x_a Z_i  (r channels; N_i square of dim d[a]; Z stack stride s)
void channel_sum(ttn_ctx* c, const cplx* Nst, const cplx* Zst, const int* d, int a, int r, cplx* Y,
                 double beta) {
    GemmArgs g = base_args();
    g.beta = C(beta);
    int d0 = d[0], d1 = d[1], d2 = d[2];
    long long s = (long long)d0 * d1 * d2;
    int D = d[a];
    long long DD = (long long)D * D;
    g.Ko = r;
    if (a == 0) {
        g.M = d0; g.N = d1 * d2; g.Ki = d0;
        g.A = Nst; g.a_m = 1; g.a_ki = D; g.a_ko = DD;
        g.B = Zst; g.b_ki = 1; g.b_ko = s; g.b_n = d0;
        g.C = Y; g.c_m = 1; g.c_n = d0;
    } else if (a == 1) {
        g.M = d0; g.N = d1; g.Ki = d1;
        g.A = Zst; g.a_m = 1; g.a_ki = d0; g.a_ko = s; g.a_bi = (long long)d0 * d1;
        g.B = Nst; g.b_ki = D; g.b_ko = DD; g.b_n = 1;
        g.C = Y; g.c_m = 1; g.c_n = d0; g.c_bi = (long long)d0 * d1;
        g.Bi = d2;
    } else {
        g.M = d0 * d1; g.N = d2; g.Ki = d2;
        g.A = Zst; g.a_m = 1; g.a_ki = (long long)d0 * d1; g.a_ko = s;
        g.B = Nst; g.b_ki = D; g.b_ko = DD; g.b_n = 1;
        g.C = Y; g.c_m = 1; g.c_n = (long long)d0 * d1;
    }
    gemm(c, g);
}

// E_i = X^H W_i contracted over every leg except o (nb stacked W, stride s;
// outputs stride d[o]^2).  Xh has dims dx, W dims dw (equal except leg o).
void project(ttn_ctx* c, const cplx* X, const int* dx, const cplx* W, const int* dw, int o, cplx* E, int nb,
             long long w_bs, long long e_bs) {
    GemmArgs g = base_args();
    g.conjA = 1;
    int x0 = dx[0], x1 = dx[1];
    if (o == 2) {
        g.M = dx[2]; g.N = dw[2]; g.Ki = x0 * x1;
        g.A = X; g.a_m = (long long)x0 * x1; g.a_ki = 1;
        g.B = W; g.b_ki = 1; g.b_n = (long long)dw[0] * dw[1];
        g.C = E; g.c_m = 1; g.c_n = dx[2];
    } else if (o == 0) {
        g.M = x0; g.N = dw[0]; g.Ki = dx[1] * dx[2];
        g.A = X; g.a_m = 1; g.a_ki = x0;
        g.B = W; g.b_ki = dw[0]; g.b_n = 1;
        g.C = E; g.c_m = 1; g.c_n = x0;
    } else {
        g.M = x1; g.N = dw[1]; g.Ki = x0; g.Ko = dx[2];
        g.A = X; g.a_m = x0; g.a_ki = 1; g.a_ko = (long long)x0 * x1;
        g.B = W; g.b_ki = 1; g.b_ko = (long long)dw[0] * dw[1]; g.b_n = dw[0];
        g.C = E; g.c_m = 1; g.c_n = x1;
    }
    g.Bi = nb; g.a_bi = 0; g.b_bi = w_bs; g.c_bi = e_bs;
    gemm(c, g);
}

// ----------------------------------------------------------- env helpers
const Env& env_of(ttn_ctx* c, int k, int leg) {
    if (leg == 2) return k == c->root ? c->dummy : c->down[k];
    int ch = c->nodes[k].child[leg];
    return ch >= 0 ? c->up[ch] : c->phys[-ch - 1];
}

// Weights of the G stack: |S_b| x |S_a|, element (j, i) = V(a_i, b_j), as
// real doubles (FP64 weighted sum) and as complex numbers (split contraction).
std::pair<double*, cplx*> vsub_for(ttn_ctx* c, const Env& a, const Env& b) {
    auto key = std::make_pair(&a, &b);
    auto it = c->vsub.find(key);
    if (it != c->vsub.end()) return it->second;
    size_t nb = b.sites.size(), na = a.sites.size();
    std::vector<double> h(nb * na);
    std::vector<cplx> hc(nb * na);
    for (size_t i = 0; i < na; ++i)
        for (size_t j = 0; j < nb; ++j) {
            h[j + nb * i] = c->V[(size_t)a.sites[i] * c->N + b.sites[j]];
            hc[j + nb * i] = C(h[j + nb * i]);
        }
    double* d = (double*)dalloc(c, sizeof(double) * std::max<size_t>(1, h.size()));
    cplx* dc = (cplx*)dalloc(c, sizeof(cplx) * std::max<size_t>(1, h.size()));
    if (!h.empty()) {
        CUDA_OK(cudaMemcpy(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(dc, hc.data(), sizeof(cplx) * hc.size(), cudaMemcpyHostToDevice));
    }
    c->vsub[key] = {d, dc};
    return c->vsub[key];
}

// G_i = sum_j V_ij n_j^(b) for every atom i of env a, into Gbuf: in split
// precision a tensor-core contraction of the n stack with the weights when it
// fills the tiles, else an FP64 weighted sum of the n stack.
void build_G(ttn_ctx* c, const Env& a, const Env& b, cplx* G) {
    int r = (int)a.sites.size(), nbs = (int)b.sites.size();
    long long DD = (long long)b.D * b.D;
    auto w = vsub_for(c, a, b);
    GemmArgs g = base_args();
    g.M = (int)DD; g.N = r; g.Ki = nbs;
    g.A = b.nops; g.a_m = 1; g.a_ki = DD;
    g.B = w.second; g.b_ki = 1; g.b_n = nbs;
    g.C = G; g.c_m = 1; g.c_n = DD;
    if (c->prec == TTN_SPLIT_TF32X3 && !g_force_fp64 && split_workspace_bytes(g) > 0) {
        gemm(c, g);
        return;
    }
    ProfScope ps(c, PK_F64, 4.0 * r * (double)nbs * DD, 0.0);
    ps.shape[0] = (int)DD; ps.shape[1] = r; ps.shape[2] = nbs; ps.shape[3] = 1;
    c->stats[3] += k_weighted_sum(b.nops, nbs, DD, w.first, r, G, c->stream);
}

// Pairs of an effective Hamiltonian over envs e[0..2]; G stacks built.
int setup_pairs(ttn_ctx* c, const Env* const* e, Pair* pairs) {
    static const int PU[3] = {0, 0, 1}, PV[3] = {1, 2, 2};
    int np = 0;
    for (int p = 0; p < 3; ++p) {
        const Env& eu = *e[PU[p]];
        const Env& ev = *e[PV[p]];
        if (eu.sites.empty() || ev.sites.empty()) continue;
        bool uside = eu.sites.size() <= ev.sites.size();
        const Env& ea = uside ? eu : ev;
        const Env& eb = uside ? ev : eu;
        Pair& P = pairs[np];
        P.a = uside ? PU[p] : PV[p];
        P.b = uside ? PV[p] : PU[p];
        P.r = (int)ea.sites.size();
        P.Na = ea.nops;
        P.G = c->Gbuf[np];
        build_G(c, ea, eb, P.G);
        ++np;
    }
    return np;
}

// Y = H_eff X with block matrices hb[u] (nullptr: zero) and channel pairs.
void heff_apply(ttn_ctx* c, const int* d, cplx* const* hb, const int* Dl, const Pair* pairs, int np,
                const cplx* X, cplx* Y) {
    double beta = 0.0;
    for (int u = 0; u < 3; ++u) {
        if (!hb[u]) continue;
        leg_apply(c, hb[u], Dl[u], X, d, u, Y, beta);
        beta = 1.0;
    }
    long long s = (long long)d[0] * d[1] * d[2];
    for (int p = 0; p < np; ++p) {
        const Pair& P = pairs[p];
        if (P.r == 0) continue;
        // Z_i = G_i x_b X for all i
        long long DDb = (long long)d[P.b] * d[P.b];
        leg_apply(c, P.G, d[P.b], X, d, P.b, c->Z, 0.0, P.r, DDb, s);
        channel_sum(c, P.Na, c->Z, d, P.a, P.r, Y, beta);
        beta = 1.0;
    }
    if (beta == 0.0) c->stats[3] += k_fill(Y, s, C(0.0), c->stream);
}

// ------------------------------------------- split-precision H_eff (a8)
// H_eff X in split precision with every operand packed once per use:
//   per leg u a stacked operand  P_u = [X | Z^(p) for each pair p with a = u]
//   (rows: the other two legs; K: the leg-u index and, per pair, the channel
//   index) and the operator stack  Q_u = [H_block(u) | n_1 .. n_r of each
//   pair]  (packed once per Krylov run), so that
//     H_eff X = sum_u Q_u x_u P_u
//   is one long-K contraction per leg.  The channel intermediates
//   Z_i = G_i x_b X are contractions whose epilogue writes TF32 planes
//   straight into the K slots of P_a (no FP64 round trip through HBM), and X
//   is packed once per leg per matvec.  Row layouts of P_u:
//     u = 0: row b + d1 c;  u = 1: row a + Pp_1 c (batch c);  u = 2: row a + d0 b.
long long grow_zeroed(ttn_ctx* c, float*& buf, size_t& cap, size_t bytes) {
    if (bytes <= cap) return 0;
    CUDA_OK(cudaStreamSynchronize(c->stream));
    if (buf) cudaFree(buf);
    buf = nullptr;
    cap = 0;
    size_t want = bytes + bytes / 8;
    if (test_take_alloc_fail() || cudaMalloc(&buf, want) != cudaSuccess) {
        buf = nullptr;
        throw TtnError(TTN_ERR_ALLOC, "split operand planes");
    }
    CUDA_OK(cudaMemsetAsync(buf, 0, want, c->stream));
    cap = want;
    return 1;
}

struct SplitHeff {
    struct Leg {
        bool on = false;      // X is packed on this leg (it has terms or feeds a channel)
        bool terms = false;   // the leg carries a block term or channel sums
        int d = 0;            // leg dimension
        int Pn = 0, Pp = 0;   // valid / padded P rows per batch
        int nb = 1;           // row batches (d2 for leg 1)
        long long rows = 0;   // P rows in the planes
        int Kc = 0, Kp = 0;   // complex K of the stack, floats per row
        int Qrows = 0;        // padded real rows of the operator stack
        int nslots = 0;       // complex K used so far while laying out
        float *Ph = nullptr, *Pl = nullptr, *Qh = nullptr, *Ql = nullptr;
    } leg[3];
    struct PairPlan {
        int a, b, r;
        long long base;       // complex K offset of the pair's slot in P_a
        int Kz;               // K' of the G contraction (floats)
        int Qrows;            // padded real rows of one G matrix
        float *Gh = nullptr, *Gl = nullptr;
        // transposed pairs (a later than b, except (1, 0)): X packed with
        // leg a's index fastest, so the epilogue's stores are coalesced
        bool trans = false;
        int Xrows = 0, XPp = 0;
        float *Xh = nullptr, *Xl = nullptr;
    } pp[3];
    int np = 0;
    int d[3] = {0, 0, 0};
    bool ok = false;
};

bool split_heff_prepare(ttn_ctx* c, SplitHeff& S, const int* d, cplx* const* hb, const Pair* pairs, int np) {
    S = SplitHeff();
    if (c->prec != TTN_SPLIT_TF32X3 || g_force_fp64) return false;
    for (int u = 0; u < 3; ++u) S.d[u] = d[u];
    for (int u = 0; u < 3; ++u) {
        SplitHeff::Leg& L = S.leg[u];
        L.terms = hb[u] != nullptr;
        for (int p = 0; p < np; ++p)
            if (pairs[p].a == u) L.terms = true;
        L.on = L.terms;
        for (int p = 0; p < np; ++p)
            if (pairs[p].b == u) L.on = true;
        if (!L.on) continue;
        L.d = d[u];
        if (u == 0) {
            L.Pn = d[1] * d[2];
        } else if (u == 1) {
            L.Pn = d[0];
            L.nb = d[2];
        } else {
            L.Pn = d[0] * d[1];
        }
        // tile efficiency: the operator side needs at least 16 rows and the
        // stacked side at least 64 rows (else the FP64 kernel is as fast)
        if (L.d < 16 || (long long)L.Pn * L.nb < 64) return false;
        L.Pp = (int)((L.Pn + SPLIT_BM - 1) / SPLIT_BM * SPLIT_BM);
        L.rows = (long long)L.Pp * L.nb;
        L.Kc = L.d;   // slot 0: X
        L.Qrows = (2 * L.d + SPLIT_BN - 1) / SPLIT_BN * SPLIT_BN;
    }
    if (!S.leg[0].on && !S.leg[1].on && !S.leg[2].on) return false;
    S.np = np;
    for (int p = 0; p < np; ++p) {
        SplitHeff::PairPlan& P = S.pp[p];
        P.a = pairs[p].a;
        P.b = pairs[p].b;
        P.r = pairs[p].r;
        P.base = S.leg[P.a].Kc;
        S.leg[P.a].Kc += S.leg[P.a].d * P.r;
        P.Kz = (2 * d[P.b] + SPLIT_BK - 1) / SPLIT_BK * SPLIT_BK;
        P.Qrows = S.leg[P.b].Qrows;
        P.trans = (P.a == 2 && P.b == 0) || (P.a == 2 && P.b == 1) || (P.a == 1 && P.b == 2);
        if (P.trans) {
            P.Xrows = P.b == 0 ? d[1] * d[2] : P.b == 1 ? d[0] * d[2] : d[0] * d[1];
            P.XPp = (P.Xrows + SPLIT_BM - 1) / SPLIT_BM * SPLIT_BM;
        }
    }
    for (int u = 0; u < 3; ++u) {
        SplitHeff::Leg& L = S.leg[u];
        if (!L.on) continue;
        L.Kp = (2 * L.Kc + SPLIT_BK - 1) / SPLIT_BK * SPLIT_BK;
        const size_t pe = (size_t)L.rows * L.Kp, qe = (size_t)L.Qrows * L.Kp;
        grow_zeroed(c, c->shP[u], c->shP_cap[u], 2 * pe * sizeof(float));
        grow_zeroed(c, c->shQ[u], c->shQ_cap[u], 2 * qe * sizeof(float));
        L.Ph = c->shP[u];
        L.Pl = L.Ph + pe;
        L.Qh = c->shQ[u];
        L.Ql = L.Qh + qe;
    }
    for (int p = 0; p < np; ++p) {
        SplitHeff::PairPlan& P = S.pp[p];
        const size_t ge = (size_t)P.r * P.Qrows * P.Kz;
        grow_zeroed(c, c->shG[p], c->shG_cap[p], 2 * ge * sizeof(float));
        P.Gh = c->shG[p];
        P.Gl = P.Gh + ge;
        if (P.trans) {
            const size_t xe = (size_t)P.XPp * P.Kz;
            grow_zeroed(c, c->shX[p], c->shX_cap[p], 2 * xe * sizeof(float));
            P.Xh = c->shX[p];
            P.Xl = P.Xh + xe;
        }
    }
    // operator stacks Q_u = [H_block(u) | n stacks of the pairs with a = u]
    auto pack_ops = [&](SplitHeff::Leg& L, const cplx* src, int nmat, long long k_off_c, int Kc_write) {
        SplitPackArgs a;
        std::memset(&a, 0, sizeof(a));
        a.src = src;
        a.R = src ? L.d : 0;
        a.Ki = L.d;
        a.Ko = std::max(1, nmat);
        a.s_r = 1;
        a.s_ki = L.d;
        a.s_ko = (long long)L.d * L.d;
        a.Bi = a.Bo = 1;
        a.embed = 1;
        a.Rpad = L.Qrows / 2;
        a.Kc = Kc_write;
        a.pitch = L.Kp;
        a.k_off = 2 * k_off_c;
        a.hi = L.Qh;
        a.lo = L.Ql;
        c->stats[3] += split_pack(a, c->stream);
    };
    for (int u = 0; u < 3; ++u) {
        SplitHeff::Leg& L = S.leg[u];
        if (!L.on) continue;
        if (hb[u]) pack_ops(L, hb[u], 1, 0, L.d);
        else pack_ops(L, nullptr, 1, 0, L.d);   // no block term: zero slot
        for (int p = 0; p < np; ++p)
            if (S.pp[p].a == u) pack_ops(L, pairs[p].Na, S.pp[p].r, S.pp[p].base, L.d * S.pp[p].r);
        if (L.Kp > 2 * L.Kc) pack_ops(L, nullptr, 1, L.Kc, (L.Kp - 2 * L.Kc) / 2);   // K padding
    }
    // G stacks: the operator side of Z_i = G_i x_b X, one padded block per i
    for (int p = 0; p < np; ++p) {
        SplitHeff::PairPlan& P = S.pp[p];
        SplitPackArgs a;
        std::memset(&a, 0, sizeof(a));
        const int db = d[P.b];
        a.src = pairs[p].G;
        a.R = db;
        a.Ki = db;
        a.Ko = 1;
        a.s_r = 1;
        a.s_ki = db;
        a.Bi = P.r;
        a.s_bi = (long long)db * db;
        a.Bo = 1;
        a.embed = 1;
        a.Rpad = P.Qrows / 2;
        a.Kc = P.Kz / 2;
        a.rb_i = P.Qrows;
        a.pitch = P.Kz;
        a.hi = P.Gh;
        a.lo = P.Gl;
        c->stats[3] += split_pack(a, c->stream);
    }
    S.ok = true;
    return true;
}

int* split_flag(ttn_ctx* c) {
    if (c->split_cap < 256) grow_split_ws(c, 256);
    return reinterpret_cast<int*>(c->split_ws);
}

// y = H_eff x with the prepared stacks.
void split_heff_apply(ttn_ctx* c, const SplitHeff& S, const cplx* x, cplx* y) {
    const int d0 = S.d[0], d1 = S.d[1], d2 = S.d[2];
    int* flag = split_flag(c);
    // 1. X into slot 0 of every stacked operand
    for (int u = 0; u < 3; ++u) {
        const SplitHeff::Leg& L = S.leg[u];
        if (!L.on) continue;
        SplitPackArgs a;
        std::memset(&a, 0, sizeof(a));
        a.src = x;
        a.Ko = 1;
        a.Bi = a.Bo = 1;
        if (u == 0) {
            a.R = d1 * d2; a.s_r = d0; a.Ki = d0; a.s_ki = 1;
        } else if (u == 1) {
            a.R = d0; a.s_r = 1; a.Ki = d1; a.s_ki = d0; a.Bi = d2; a.s_bi = (long long)d0 * d1; a.rb_i = L.Pp;
        } else {
            a.R = d0 * d1; a.s_r = 1; a.Ki = d2; a.s_ki = (long long)d0 * d1;
        }
        a.Rpad = a.R;
        a.Kc = L.d;
        a.pitch = L.Kp;
        a.hi = L.Ph;
        a.lo = L.Pl;
        ProfScope ps(c, PK_PACK, 0.0, (double)a.R * a.Bi * L.d * 32.0);
        c->stats[3] += split_pack(a, c->stream);
    }
    // 2. channel intermediates Z_i = G_i x_b X, written into the K slots of P_a
    const int BIG = 1 << 30;
    for (int p = 0; p < S.np; ++p) {
        const SplitHeff::PairPlan& P = S.pp[p];
        const SplitHeff::Leg& Lb = S.leg[P.b];
        const SplitHeff::Leg& La = S.leg[P.a];
        const long long K2 = La.Kp / 2;
        const int a = P.a, b = P.b;
        SplitMma m;
        std::memset(&m, 0, sizeof(m));
        m.Qh = P.Gh; m.Ql = P.Gl; m.Q_rows = (long long)P.r * P.Qrows; m.Q_pitch = P.Kz;
        m.Kp = P.Kz;
        m.Qn = Lb.d; m.Qp = P.Qrows;
        m.alpha = C(1.0);
        m.beta = C(0.0);
        m.max_split = 1;
        SplitOut o;
        std::memset(&o, 0, sizeof(o));
        o.hi = La.Ph + 2 * P.base;
        o.lo = La.Pl + 2 * P.base;
        o.pd = BIG;
        o.sp1 = 1;
        if (P.trans) {
            // X with leg a's index fastest: rows (x fastest, then y), K = leg b
            SplitPackArgs xa;
            std::memset(&xa, 0, sizeof(xa));
            xa.src = x;
            xa.Ko = 1;
            xa.Bo = 1;
            if (b == 0) {          // (a, b) = (2, 0): rows c + d2 b'
                xa.R = d2; xa.s_r = (long long)d0 * d1; xa.Bi = d1; xa.s_bi = d0; xa.Ki = d0; xa.s_ki = 1;
            } else if (b == 1) {   // (2, 1): rows c + d2 a
                xa.R = d2; xa.s_r = (long long)d0 * d1; xa.Bi = d0; xa.s_bi = 1; xa.Ki = d1; xa.s_ki = d0;
            } else {               // (1, 2): rows b + d1 a
                xa.R = d1; xa.s_r = d0; xa.Bi = d0; xa.s_bi = 1; xa.Ki = d2; xa.s_ki = (long long)d0 * d1;
            }
            xa.Rpad = xa.R;
            xa.rb_i = xa.R;
            xa.Kc = S.d[b];
            xa.pitch = P.Kz;
            xa.hi = P.Xh;
            xa.lo = P.Xl;
            {
                ProfScope ps(c, PK_PACK, 0.0, (double)xa.R * xa.Bi * S.d[b] * 32.0);
                c->stats[3] += split_pack(xa, c->stream);
            }
            m.Ph = P.Xh; m.Pl = P.Xl; m.P_rows = P.XPp; m.P_pitch = P.Kz;
            m.Pn = P.Xrows; m.Pp = P.XPp;
            m.Bi = P.r; m.Bo = 1; m.q_sbi = P.Qrows;
            o.sbi = S.d[a];
            if (b == 0) {
                o.pd = d2; o.sp2 = (long long)d0 * K2; o.sq = K2;
            } else if (b == 1) {
                o.pd = d2; o.sp2 = K2; o.sq = (long long)d0 * K2;
            } else {
                o.pd = d1; o.sp2 = K2; o.sq = (long long)La.Pp * K2;
            }
        } else {
            m.Ph = Lb.Ph; m.Pl = Lb.Pl; m.P_rows = Lb.rows; m.P_pitch = Lb.Kp;
            m.Pn = Lb.Pn; m.Pp = Lb.Pp;
            if (b == 1) {          // (0, 1): p = a, bi = c, q = b', bo = i
                m.Bi = d2; m.Bo = P.r; m.p_sbi = Lb.Pp; m.q_sbo = P.Qrows;
                o.sq = K2; o.sbi = (long long)d1 * K2; o.sbo = d0;
            } else {
                m.Bi = P.r; m.Bo = 1; m.q_sbi = P.Qrows;
                if (b == 2) {      // (0, 2): p = a + d0 b, q = c', bi = i
                    o.pd = d0; o.sp2 = K2; o.sq = (long long)d1 * K2; o.sbi = d0;
                } else {           // (1, 0): p = b + d1 c, q = a', bi = i
                    o.pd = d1; o.sp2 = (long long)La.Pp * K2; o.sq = K2; o.sbi = d1;
                }
            }
        }
        m.out = &o;
        const double fl = 8.0 * (double)m.Pn * m.Bi * m.Bo * Lb.d * Lb.d;
        ProfScope ps(c, PK_TC, fl, 0.0);
        ps.shape[0] = m.Pn; ps.shape[1] = Lb.d; ps.shape[2] = Lb.d; ps.shape[3] = m.Bi * m.Bo;
        int n = split_mma(m, flag, nullptr, 0, c->stream);
        if (n < 0) throw TtnError(TTN_ERR_CUDA, "split channel contraction launch failed");
        c->stats[3] += n;
    }
    // 3. one long-K contraction per leg: Y (+)= Q_u x_u P_u
    bool first = true;
    for (int u = 0; u < 3; ++u) {
        const SplitHeff::Leg& L = S.leg[u];
        if (!L.terms) continue;
        SplitMma m;
        std::memset(&m, 0, sizeof(m));
        m.Ph = L.Ph; m.Pl = L.Pl; m.P_rows = L.rows; m.P_pitch = L.Kp;
        m.Qh = L.Qh; m.Ql = L.Ql; m.Q_rows = L.Qrows; m.Q_pitch = L.Kp;
        m.Kp = L.Kp;
        m.Pn = L.Pn; m.Pp = L.Pp;
        m.Qn = L.d; m.Qp = L.Qrows;
        m.Bi = L.nb; m.Bo = 1;
        m.p_sbi = u == 1 ? L.Pp : 0;
        m.C = y;
        if (u == 0) {
            m.c_p = d0; m.c_q = 1;
        } else if (u == 1) {
            m.c_p = 1; m.c_q = d0; m.c_bi = (long long)d0 * d1;
        } else {
            m.c_p = 1; m.c_q = (long long)d0 * d1;
        }
        m.alpha = C(1.0);
        m.beta = C(first ? 0.0 : 1.0);
        m.max_split = SPLIT_K_MAX;
        const size_t pb = split_mma_partials(m);
        if (c->split_cap < 256 + pb) grow_split_ws(c, 256 + pb);
        flag = reinterpret_cast<int*>(c->split_ws);
        const double fl = 8.0 * (double)L.Pn * L.nb * L.d * L.Kc;
        ProfScope ps(c, PK_TC, fl, 0.0);
        ps.shape[0] = L.Pn; ps.shape[1] = L.d; ps.shape[2] = L.Kc; ps.shape[3] = L.nb;
        int n = split_mma(m, flag, reinterpret_cast<uint8_t*>(c->split_ws) + 256, c->split_cap - 256, c->stream);
        if (n < 0) throw TtnError(TTN_ERR_CUDA, "split stacked contraction launch failed");
        c->stats[3] += n;
        first = false;
    }
    if (first) c->stats[3] += k_fill(y, (long long)d0 * d1 * d2, C(0.0), c->stream);
}

void assemble(ttn_ctx* c, const Env& e, cplx* out) {
    ProfScope ps(c, PK_MISC, 0.0, 0.0);
    c->stats[3] += k_assemble_block(out, e.has_H ? e.H : nullptr, e.D, e.nops, (int)e.sites.size(),
                                    e.d_sites, e.dops, (int)e.driven.size(), e.d_driven, c->d_coef, c->gamma,
                                    c->stream);
}

bool env_has_block(const Env& e) { return e.has_H || !e.sites.empty(); }

// --------------------------------------------------------------- Krylov
// x <- exp(z H) x with H given by `apply`, Lanczos with full two-pass
// re-orthogonalisation; z = (zr, zi).
template <class F>
void krylov(ttn_ctx* c, cplx* x, long long n, double zr, double zi, F apply) {
    cudaStream_t s = c->stream;
    const double tol = (c->prec == TTN_FP64) ? 1e-13 : 1e-9;
    const int mmax = test_krylov_mmax();
    cplx* V = c->Kbasis;
    const long long ld = n;
    {
        ProfScope ps(c, PK_KRY, 0.0, 48.0 * n);
        c->stats[3] += k_norm2_partial(x, n, c->kpn, s);
        c->stats[3] += k_krylov_start_ex(c->ks, c->kpn, n, s);
        c->stats[3] += k_scale_copy_dev(x, n, &c->ks->inv_scale, V, s);
    }
    int j = 0;
    for (;; ++j) {
        cplx* vj = V + (long long)j * ld;
        cplx* w = V + (long long)(j + 1) * ld;
        apply(vj, w);
        c->stats[1] += 1;
        {
            // bytes: the basis is read three times (dots, two update passes), w read and written twice
            ProfScope ps(c, PK_KRY, 0.0, 16.0 * n * (3.0 * (j + 1) + 5.0));
            c->stats[3] += k_dots_scaled(V, ld, j + 1, w, n, c->kpart, -1, nullptr, -1, s);
            cplx* part2 = c->kpart + (size_t)RED_BLOCKS * (KRYLOV_MMAX + 1);
            c->stats[3] += k_orth_update_ex(V, ld, j + 1, c->kpart, w, n, 1, part2, nullptr, c->kh1, 0, -1, s);
            c->stats[3] += k_orth_update_ex(V, ld, j + 1, part2, w, n, 2, nullptr, c->kpn, c->kh2, 0, -1, s);
            if (c->gamma != 0.0)   // non-Hermitian generator (decay): Arnoldi
                c->stats[3] += k_arnoldi_scalars(c->ks, c->kh1, c->kh2, c->kpn, n, j, zr, zi, tol, s);
            else
                c->stats[3] += k_krylov_scalars_ex(c->ks, c->kh1, c->kh2, c->kpn, n, j, zr, zi, tol, s);
        }
        CUDA_OK(cudaMemcpyAsync(c->hflag, &c->ks->converged, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        c->hflag[2] = 0;
        if (c->split_ws)   // a tensor-core wait that gave up leaves garbage: report it first
            CUDA_OK(cudaMemcpyAsync(c->hflag + 2, c->split_ws, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
        if (c->hflag[2]) check_split_flag(c);
        if (c->hflag[1]) throw TtnError(TTN_ERR_NUMERIC, "non-finite value in Lanczos");
        if (c->hflag[0] || j == mmax - 1) break;
        ProfScope ps(c, PK_KRY, 0.0, 32.0 * n);
        c->stats[3] += k_scale_copy_dev(w, n, &c->ks->inv_scale, w, s);
    }
    if (!c->hflag[0]) {
        double err;
        CUDA_OK(cudaMemcpy(&err, &c->ks->err, sizeof(double), cudaMemcpyDeviceToHost));
        c->max_err = std::max(c->max_err, err);
        if (err > 1e-6) throw TtnError(TTN_ERR_KRYLOV, "Lanczos did not converge in m_max steps");
    }
    c->stats[0] += 1;
    ProfScope ps(c, PK_KRY, 0.0, 16.0 * n * (j + 2));
    c->stats[3] += k_combine(V, ld, j + 1, c->ks, x, n, s);
}

// Small nodes and links (s <= SMALL_S): H_eff as a dense matrix and the whole
// Krylov exponential in one launch (same algorithm and stopping rule as
// krylov()), with one host round trip for the status instead of one per
// Lanczos step.
bool small_evolve(ttn_ctx* c, const int* d, cplx* const* hb, const Pair* pairs, int np, cplx* x, double zr,
                  double zi) {
    const long long s = (long long)d[0] * d[1] * d[2];
    if (s > SMALL_S) return false;
    SmallPairs pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.np = np;
    for (int p = 0; p < np; ++p) {
        pp.a[p] = pairs[p].a;
        pp.b[p] = pairs[p].b;
        pp.r[p] = pairs[p].r;
        pp.Na[p] = pairs[p].Na;
        pp.G[p] = pairs[p].G;
    }
    const double tol = (c->prec == TTN_FP64) ? 1e-13 : 1e-9;
    {
        ProfScope ps(c, PK_KRY, 0.0, 0.0);
        c->stats[3] += k_dense_heff(c->dense_H, d, hb[0], hb[1], hb[2], pp, c->stream);
        c->stats[3] += k_small_krylov(c->dense_H, (int)s, x, zr, zi, tol, test_krylov_mmax(),
                                      c->gamma != 0.0 ? 1 : 0, c->ks, c->stream);
    }
    struct {
        double alpha0;
        double err;
        int flags[2];
    } st;
    CUDA_OK(cudaMemcpyAsync(&st.alpha0, &c->ks->alpha[0], sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaMemcpyAsync(&st.err, &c->ks->err, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaMemcpyAsync(st.flags, &c->ks->converged, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    if (st.flags[1]) throw TtnError(TTN_ERR_NUMERIC, "non-finite value in Lanczos");
    c->stats[0] += 1;
    c->stats[1] += (int64_t)st.alpha0;
    if (!st.flags[0]) {
        c->max_err = std::max(c->max_err, st.err);
        if (st.err > 1e-6) throw TtnError(TTN_ERR_KRYLOV, "Lanczos did not converge in m_max steps");
    }
    return true;
}

// ------------------------------------------------------ renormalisation
void ensure_env_capacity(ttn_ctx* c, Env& E, size_t nn, size_t nd) {
    long long DD = (long long)E.D * E.D;
    if (!E.H) E.H = (cplx*)dalloc(c, sizeof(cplx) * DD);
    if (nn > E.cap_n) {
        E.nops = (cplx*)dalloc(c, sizeof(cplx) * DD * nn);
        E.d_sites = (int*)dalloc(c, sizeof(int) * nn);
        E.cap_n = nn;
    }
    if (nd > E.cap_d) {
        E.dops = (cplx*)dalloc(c, sizeof(cplx) * DD * 3 * nd);
        E.d_driven = (int*)dalloc(c, sizeof(int) * nd);
        E.cap_d = nd;
    }
}

// Split-precision renormalisation of an operator stack (a2): for every op_i
// on leg u, E_i = X^H (op_i x_u X) contracted over the legs other than o.
// The intermediate Z_i = op_i x_u X goes straight from the contraction
// epilogue into TF32 planes laid out for the projection, whose rows are
// (leg-o index, i) and whose K runs over (w, u) with w the third leg, w
// fastest (so that consecutive rows of the first contraction -- X packed with
// leg w fastest -- land next to each other).  Returns false when the shape
// does not fill the tensor-core tiles (the caller then runs the FP64 or
// generic split contractions).  Uses the H_eff planes as scratch: no Krylov
// run is in flight while environments are rebuilt.
bool renorm_stack_split(ttn_ctx* c, const cplx* X, const int* d, int u, int o, const cplx* ops, int nop,
                        cplx* out) {
    if (c->prec != TTN_SPLIT_TF32X3 || g_force_fp64 || nop < 1) return false;
    const int w = 3 - u - o;
    const int du = d[u], dO = d[o], dw = d[w];
    if (du < 16 || dO < 16 || (long long)dw * dO < 64) return false;
    const long long s = (long long)d[0] * d[1] * d[2];
    const long long st[3] = {1, d[0], (long long)d[0] * d[1]};
    const long long DDu = (long long)du * du, DDo = (long long)dO * dO;
    const int Kz = (2 * du + SPLIT_BK - 1) / SPLIT_BK * SPLIT_BK;           // K' of op x_u X
    const long long Kproj = s / dO;                                          // complex K of the projection
    const int Kp = (int)((2 * Kproj + SPLIT_BK - 1) / SPLIT_BK * SPLIT_BK);
    const int Qrows_u = (2 * du + SPLIT_BN - 1) / SPLIT_BN * SPLIT_BN;
    const int Qrows_o = (2 * dO + SPLIT_BN - 1) / SPLIT_BN * SPLIT_BN;
    const int Pz = dw * dO, Pzp = (Pz + SPLIT_BM - 1) / SPLIT_BM * SPLIT_BM;
    int chunk = (int)std::max<long long>(1, c->zcap / s);
    chunk = std::min(chunk, nop);
    const int Pproj_max = (int)((dO * (long long)chunk + SPLIT_BM - 1) / SPLIT_BM * SPLIT_BM);
    // buffers: X for the first contraction, the op stack, X^H, the projection's P side
    const size_t xe = (size_t)Pzp * Kz, oe = (size_t)nop * Qrows_u * Kz, ce = (size_t)Qrows_o * Kp,
                 pe = (size_t)Pproj_max * Kp;
    grow_zeroed(c, c->shX[0], c->shX_cap[0], 2 * xe * sizeof(float));
    grow_zeroed(c, c->shG[0], c->shG_cap[0], 2 * oe * sizeof(float));
    grow_zeroed(c, c->shQ[0], c->shQ_cap[0], 2 * ce * sizeof(float));
    grow_zeroed(c, c->shP[0], c->shP_cap[0], 2 * pe * sizeof(float));
    float *Xh = c->shX[0], *Xl = Xh + xe, *Oh = c->shG[0], *Ol = Oh + oe, *Ch = c->shQ[0], *Cl = Ch + ce,
          *Ph = c->shP[0], *Pl = Ph + pe;
    SplitPackArgs a;
    // X with rows w + dw * o-index, K = u-index
    std::memset(&a, 0, sizeof(a));
    a.src = X; a.R = dw; a.s_r = st[w]; a.Bi = dO; a.s_bi = st[o]; a.rb_i = dw; a.Bo = 1;
    a.Ki = du; a.s_ki = st[u]; a.Ko = 1; a.Rpad = dw; a.Kc = Kz / 2; a.pitch = Kz; a.hi = Xh; a.lo = Xl;
    c->stats[3] += split_pack(a, c->stream);
    // op stack, embedded: rows = new u-index, K = old u-index, one padded block per op
    std::memset(&a, 0, sizeof(a));
    a.src = ops; a.R = du; a.s_r = 1; a.Ki = du; a.s_ki = du; a.Ko = 1; a.Bi = nop; a.s_bi = DDu; a.Bo = 1;
    a.rb_i = Qrows_u; a.embed = 1; a.Rpad = Qrows_u / 2; a.Kc = Kz / 2; a.pitch = Kz; a.hi = Oh; a.lo = Ol;
    c->stats[3] += split_pack(a, c->stream);
    // X^H, embedded: rows = o-index, K = w + dw * u
    std::memset(&a, 0, sizeof(a));
    a.src = X; a.R = dO; a.s_r = st[o]; a.Ki = dw; a.s_ki = st[w]; a.Ko = du; a.s_ko = st[u]; a.Bi = a.Bo = 1;
    a.conj = 1; a.embed = 1; a.Rpad = Qrows_o / 2; a.Kc = Kp / 2; a.pitch = Kp; a.hi = Ch; a.lo = Cl;
    c->stats[3] += split_pack(a, c->stream);
    int* flag = split_flag(c);
    for (int i0 = 0; i0 < nop; i0 += chunk) {
        const int nb = std::min(chunk, nop - i0);
        // Z_i = op_i x_u X into the projection's planes: row o-index + dO i, K w + dw u'
        SplitMma m;
        std::memset(&m, 0, sizeof(m));
        m.Ph = Xh; m.Pl = Xl; m.P_rows = Pzp; m.P_pitch = Kz;
        m.Qh = Oh + (size_t)i0 * Qrows_u * Kz; m.Ql = Ol + (size_t)i0 * Qrows_u * Kz;
        m.Q_rows = (long long)nb * Qrows_u; m.Q_pitch = Kz;
        m.Kp = Kz;
        m.Pn = Pz; m.Pp = Pzp; m.Qn = du; m.Qp = Qrows_u;
        m.Bi = nb; m.Bo = 1; m.q_sbi = Qrows_u;
        m.alpha = C(1.0);
        m.beta = C(0.0);
        m.max_split = 1;
        SplitOut so;
        std::memset(&so, 0, sizeof(so));
        const long long K2 = Kp / 2;
        so.hi = Ph; so.lo = Pl; so.pd = dw; so.sp1 = 1; so.sp2 = K2; so.sq = dw; so.sbi = (long long)dO * K2;
        m.out = &so;
        {
            ProfScope ps(c, PK_TC, 8.0 * (double)Pz * du * du * nb, 0.0);
            ps.shape[0] = Pz; ps.shape[1] = du; ps.shape[2] = du; ps.shape[3] = nb;
            int n = split_mma(m, flag, nullptr, 0, c->stream);
            if (n < 0) throw TtnError(TTN_ERR_CUDA, "split renormalisation launch failed");
            c->stats[3] += n;
        }
        // E_i(k, k') = sum conj(X(..k..)) Z_i(..k'..): P rows k' + dO i, Q rows k
        SplitMma pj;
        std::memset(&pj, 0, sizeof(pj));
        const int Pn = dO * nb, Pp = (Pn + SPLIT_BM - 1) / SPLIT_BM * SPLIT_BM;
        pj.Ph = Ph; pj.Pl = Pl; pj.P_rows = Pp; pj.P_pitch = Kp;
        pj.Qh = Ch; pj.Ql = Cl; pj.Q_rows = Qrows_o; pj.Q_pitch = Kp;
        pj.Kp = Kp;
        pj.Pn = Pn; pj.Pp = Pp; pj.Qn = dO; pj.Qp = Qrows_o;
        pj.Bi = pj.Bo = 1;
        pj.C = out + (long long)i0 * DDo;
        pj.c_pd = dO; pj.c_p = dO; pj.c_p2 = DDo; pj.c_q = 1;
        pj.alpha = C(1.0);
        pj.beta = C(0.0);
        pj.max_split = SPLIT_K_MAX;
        const size_t pb = split_mma_partials(pj);
        if (c->split_cap < 256 + pb) grow_split_ws(c, 256 + pb);
        flag = reinterpret_cast<int*>(c->split_ws);
        ProfScope ps(c, PK_TC, 8.0 * (double)Pn * dO * Kproj, 0.0);
        ps.shape[0] = Pn; ps.shape[1] = dO; ps.shape[2] = (int)Kproj; ps.shape[3] = 1;
        int n = split_mma(pj, flag, reinterpret_cast<uint8_t*>(c->split_ws) + 256, c->split_cap - 256, c->stream);
        if (n < 0) throw TtnError(TTN_ERR_CUDA, "split projection launch failed");
        c->stats[3] += n;
    }
    return true;
}

// op stack (nop matrices of D_u^2) on leg u of X -> projected stack on leg o
void renorm_stack(ttn_ctx* c, const cplx* X, const int* d, int u, int o, const cplx* ops, int nop, cplx* out) {
    if (nop < 1) return;
    if (renorm_stack_split(c, X, d, u, o, ops, nop, out)) return;
    long long s = (long long)d[0] * d[1] * d[2];
    long long DDu = (long long)d[u] * d[u], DDo = (long long)d[o] * d[o];
    int chunk = (int)std::max<long long>(1, c->zcap / s);
    for (int i0 = 0; i0 < nop; i0 += chunk) {
        int nb = std::min(chunk, nop - i0);
        leg_apply(c, ops + i0 * DDu, d[u], X, d, u, c->Z, 0.0, nb, DDu, s);
        project(c, X, d, c->Z, d, o, out + i0 * DDo, nb, s, DDo);
    }
}

// Environment seen through leg o of node tensor X (isometric w.r.t. o) from
// the environments eu, ev of its other legs u < v.
void renormalize(ttn_ctx* c, const cplx* X, const int* d, int o, const Env& eu, const Env& ev, Env& E) {
    int u = (o == 0) ? 1 : 0, v = (o == 2) ? 1 : 2;
    E.D = d[o];
    E.sites = eu.sites;
    E.sites.insert(E.sites.end(), ev.sites.begin(), ev.sites.end());
    E.driven = eu.driven;
    E.driven.insert(E.driven.end(), ev.driven.begin(), ev.driven.end());
    ensure_env_capacity(c, E, E.sites.size(), E.driven.size());
    long long DDo = (long long)E.D * E.D;
    cudaStream_t s = c->stream;
    if (!E.sites.empty())
        CUDA_OK(cudaMemcpyAsync(E.d_sites, E.sites.data(), sizeof(int) * E.sites.size(), cudaMemcpyHostToDevice, s));
    if (!E.driven.empty())
        CUDA_OK(cudaMemcpyAsync(E.d_driven, E.driven.data(), sizeof(int) * E.driven.size(), cudaMemcpyHostToDevice, s));
    // static block: X^H (Hs_u + Hs_v + sum V n n) X
    const Env* e3[3];
    e3[u] = &eu;
    e3[v] = &ev;
    e3[o] = &c->dummy;
    cplx* hbs[3] = {nullptr, nullptr, nullptr};
    int Dl[3] = {d[0], d[1], d[2]};
    if (eu.has_H) hbs[u] = eu.H;
    if (ev.has_H) hbs[v] = ev.H;
    Pair pairs[3];
    int np = 0;
    if (!eu.sites.empty() && !ev.sites.empty()) {
        // only the (u, v) pair
        bool uside = eu.sites.size() <= ev.sites.size();
        const Env& ea = uside ? eu : ev;
        const Env& eb = uside ? ev : eu;
        pairs[0].a = uside ? u : v;
        pairs[0].b = uside ? v : u;
        pairs[0].r = (int)ea.sites.size();
        pairs[0].Na = ea.nops;
        pairs[0].G = c->Gbuf[0];
        build_G(c, ea, eb, pairs[0].G);
        np = 1;
    }
    (void)e3;
    E.has_H = (hbs[u] || hbs[v] || np > 0);
    if (E.has_H) {
        cplx* W = c->tmp[2];
        SplitHeff S;
        if (split_heff_prepare(c, S, d, hbs, pairs, np)) split_heff_apply(c, S, X, W);
        else heff_apply(c, d, hbs, Dl, pairs, np, X, W);
        project(c, X, d, W, d, o, E.H, 1, 0, 0);
    }
    // one-site operators
    renorm_stack(c, X, d, u, o, eu.nops, (int)eu.sites.size(), E.nops);
    renorm_stack(c, X, d, v, o, ev.nops, (int)ev.sites.size(), E.nops + eu.sites.size() * DDo);
    renorm_stack(c, X, d, u, o, eu.dops, 3 * (int)eu.driven.size(), E.dops);
    renorm_stack(c, X, d, v, o, ev.dops, 3 * (int)ev.driven.size(), E.dops + 3 * eu.driven.size() * DDo);
}

void build_up(ttn_ctx* c, int k) {
    const Node& nd = c->nodes[k];
    renormalize(c, c->T[k], nd.d, 2, env_of(c, k, 0), env_of(c, k, 1), c->up[k]);
}

void build_down(ttn_ctx* c, int k, int leg) {
    int ch = c->nodes[k].child[leg];
    int other = 1 - leg;
    const Env& e_other = env_of(c, k, other);
    const Env& e_par = env_of(c, k, 2);
    renormalize(c, c->T[k], c->nodes[k].d, leg, leg == 0 ? e_other : e_other, e_par, c->down[ch]);
}

void rebuild_up_envs(ttn_ctx* c) {
    for (auto& lev : c->level_nodes)
        for (int k : lev)
            if (k != c->root) build_up(c, k);
}

// ----------------------------------------------------------- QR & moves
// X (node k) = Q x_o R; Q replaces the node tensor, R (D x D) into Rbuf.
void qr_leg(ttn_ctx* c, int k, int o) {
    const Node& nd = c->nodes[k];
    int D = nd.d[o];
    long long s = nd.s, M = s / D;
    cplx* A = c->T[k];
    static const int PERM[3][3] = {{1, 2, 0}, {0, 2, 1}, {0, 1, 2}};
    if (o != 2) {
        ProfScope ps(c, PK_MISC, 0.0, 32.0 * nd.s);
        c->stats[3] += k_permute3(c->T[k], c->tmp[0], nd.d[0], nd.d[1], nd.d[2], PERM[o][0], PERM[o][1],
                                  PERM[o][2], 0, c->stream);
        A = c->tmp[0];
    }
    int ndep = 0;
    auto key = std::make_pair(k, o);
    {
        ProfScope ps(c, PK_QR, 16.0 * (double)M * D * D, 0.0);
        int nl = qr_cgs2(A, (int)M, D, c->Rbuf, c->cand[key], c->ncand[key], c->qr, c->stream, &ndep);
        if (nl < 0) throw TtnError(TTN_ERR_TIMEOUT, "QR grid barrier wait timed out");
        c->stats[3] += nl;
        ps.shape[0] = (int)M;   // profile record: rows, columns, dependent columns
        ps.shape[1] = D;
        ps.shape[2] = ndep;
        ps.shape[3] = 1;
    }
    c->stats[4] += 1;
    c->stats[5] += ndep;
    if (o != 2) {
        ProfScope ps(c, PK_MISC, 0.0, 32.0 * nd.s);
        c->stats[3] += k_permute3(c->tmp[0], c->T[k], nd.d[0], nd.d[1], nd.d[2], PERM[o][0], PERM[o][1],
                                  PERM[o][2], 1, c->stream);
    }
}

// node k <- Rbuf x_leg node k   (absorb the link matrix).
// Node k is an isometry from leg `leg` to its other two legs here (it was
// just QR'd towards this link), so the new centre's norm equals |R|_F in
// exact arithmetic.  In split precision the contraction's norm error is what
// drifts the state's norm (a plain split absorb lost ~1e-5 per step); the
// product is therefore rescaled to |R|_F with FP64 reductions, leaving only
// its direction error (~5e-7 relative, a second-order infidelity).  In FP64
// mode, and for gauge-only moves (`gauge_only`: observables must not perturb
// the state they read), the absorb is a plain FP64 contraction.
void absorb(ttn_ctx* c, int k, int leg, bool gauge_only = false) {
    const Node& nd = c->nodes[k];
    const long long D = nd.d[leg];
    if (c->prec == TTN_SPLIT_TF32X3 && !g_force_fp64 && !gauge_only) {
        c->stats[3] += k_norm2_partial(c->Rbuf, D * D, c->apr, c->stream);
        leg_apply(c, c->Rbuf, nd.d[leg], c->T[k], nd.d, leg, c->tmp[1], 0.0);
        ProfScope ps(c, PK_MISC, 0.0, 48.0 * nd.s);
        c->stats[3] += k_norm2_partial(c->tmp[1], nd.s, c->apx, c->stream);
        c->stats[3] += k_rescale_to_norm(c->tmp[1], nd.s, c->apx, red_blocks_for(nd.s), c->apr,
                                         red_blocks_for(D * D), c->stream);
    } else {
        ForceFp64 f64;
        leg_apply(c, c->Rbuf, nd.d[leg], c->T[k], nd.d, leg, c->tmp[1], 0.0);
    }
    std::swap(c->T[k], c->tmp[1]);
}

void node_evolve(ttn_ctx* c, int k, double tau) {
    const Node& nd = c->nodes[k];
    const Env* e[3] = {&env_of(c, k, 0), &env_of(c, k, 1), &env_of(c, k, 2)};
    cplx* hbs[3];
    int Dl[3] = {nd.d[0], nd.d[1], nd.d[2]};
    for (int u = 0; u < 3; ++u) {
        hbs[u] = nullptr;
        if (env_has_block(*e[u])) {
            assemble(c, *e[u], c->hb[u]);
            hbs[u] = c->hb[u];
        }
    }
    Pair pairs[3];
    int np = setup_pairs(c, e, pairs);
    if (small_evolve(c, nd.d, hbs, pairs, np, c->T[k], 0.0, -tau)) return;
    SplitHeff S;
    const bool sp = split_heff_prepare(c, S, nd.d, hbs, pairs, np);
    krylov(c, c->T[k], nd.s, 0.0, -tau, [&](const cplx* x, cplx* y) {
        if (sp) split_heff_apply(c, S, x, y);
        else heff_apply(c, nd.d, hbs, Dl, pairs, np, x, y);
    });
}

// R <- exp(+i tau H_link) R, rows in basis of er, columns of ec
void link_evolve(ttn_ctx* c, const Env& er, const Env& ec, double tau) {
    int d[3] = {er.D, ec.D, 1};
    const Env* e[3] = {&er, &ec, &c->dummy};
    cplx* hbs[3] = {nullptr, nullptr, nullptr};
    int Dl[3] = {d[0], d[1], 1};
    for (int u = 0; u < 2; ++u)
        if (env_has_block(*e[u])) {
            assemble(c, *e[u], c->hb[u]);
            hbs[u] = c->hb[u];
        }
    Pair pairs[3];
    int np = setup_pairs(c, e, pairs);
    if (small_evolve(c, d, hbs, pairs, np, c->Rbuf, 0.0, tau)) return;
    SplitHeff S;
    const bool sp = split_heff_prepare(c, S, d, hbs, pairs, np);
    krylov(c, c->Rbuf, (long long)d[0] * d[1], 0.0, tau, [&](const cplx* x, cplx* y) {
        if (sp) split_heff_apply(c, S, x, y);
        else heff_apply(c, d, hbs, Dl, pairs, np, x, y);
    });
}

std::vector<std::pair<int, int>> node_children(const ttn_ctx* c, int k) {
    std::vector<std::pair<int, int>> out;
    for (int u = 0; u < 2; ++u)
        if (c->nodes[k].child[u] >= 0) out.push_back({u, c->nodes[k].child[u]});
    return out;
}

void sweep_fwd(ttn_ctx* c, int k, double tau) {
    for (auto [u, ch] : node_children(c, k)) {
        qr_leg(c, k, u);
        build_down(c, k, u);
        absorb(c, ch, 2);
        sweep_fwd(c, ch, tau);
        qr_leg(c, ch, 2);
        build_up(c, ch);
        link_evolve(c, c->up[ch], c->down[ch], tau);
        absorb(c, k, u);
    }
    node_evolve(c, k, tau);
}

void sweep_rev(ttn_ctx* c, int k, double tau) {
    node_evolve(c, k, tau);
    auto ch_list = node_children(c, k);
    for (auto it = ch_list.rbegin(); it != ch_list.rend(); ++it) {
        auto [u, ch] = *it;
        qr_leg(c, k, u);
        build_down(c, k, u);
        link_evolve(c, c->down[ch], c->up[ch], tau);
        absorb(c, ch, 2);
        sweep_rev(c, ch, tau);
        qr_leg(c, ch, 2);
        build_up(c, ch);
        absorb(c, k, u);
    }
}

// Move the orthogonality centre from the root down to node k (gauge only).
void centre_to(ttn_ctx* c, int k) {
    std::vector<int> path;
    for (int x = k; x != c->root; x = c->nodes[x].parent) path.push_back(x);
    std::reverse(path.begin(), path.end());
    int cur = c->root;
    for (int ch : path) {
        int u = c->nodes[cur].child[0] == ch ? 0 : 1;
        qr_leg(c, cur, u);
        build_down(c, cur, u);
        absorb(c, ch, 2, true);
        cur = ch;
    }
    c->centre = k;
}

void centre_to_root(ttn_ctx* c) {
    if (c->centre == c->root || c->centre < 0) {
        c->centre = c->root;
        return;
    }
    int cur = c->centre;
    while (cur != c->root) {
        int par = c->nodes[cur].parent;
        int u = c->nodes[par].child[0] == cur ? 0 : 1;
        qr_leg(c, cur, 2);
        build_up(c, cur);
        absorb(c, par, u, true);
        cur = par;
    }
    c->centre = c->root;
}

// ---------------------------------------------------------------- setup
void compute_coef(ttn_ctx* c, double t) {
    std::fill(c->h_coef.begin(), c->h_coef.end(), 0.0);
    for (const ttn_pulse& p : c->schedule) {
        if (p.t0 <= t && t < p.t1) {
            double* q = &c->h_coef[5 * p.atom];
            q[0] += p.omega_x;
            q[1] += p.omega_z;
            q[2] += p.omega_r * std::cos(p.phase_r);
            q[3] += p.omega_r * std::sin(p.phase_r);
            q[4] += p.delta;
        }
    }
    CUDA_OK(cudaMemcpyAsync(c->d_coef, c->h_coef.data(), sizeof(double) * c->h_coef.size(),
                            cudaMemcpyHostToDevice, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));   // h_coef is reused on the next call
}

void set_phys_envs(ttn_ctx* c) {
    static const double NR[9] = {0, 0, 0, 0, 0, 0, 0, 0, 1};
    for (int l = 0; l < c->n_leaves; ++l) {
        Env& E = c->phys[l];
        E.D = 3;
        E.has_H = false;
        int a = c->leaf_atom[l];
        E.sites.clear();
        E.driven.clear();
        if (a < 0) continue;
        E.sites.push_back(a);
        if (c->driven[a]) E.driven.push_back(a);
        ensure_env_capacity(c, E, 1, 1);
        // column-major 3x3: element (r, col) at r + 3 col
        cplx n[9], ops[27];
        for (int i = 0; i < 9; ++i) n[i] = C(NR[i]);
        for (int i = 0; i < 27; ++i) ops[i] = C(0.0);
        ops[1 + 3 * 0] = C(1.0);  // sx: |1><0|
        ops[0 + 3 * 1] = C(1.0);  // sx: |0><1|
        ops[9 + 0] = C(1.0);      // sz (0,0)
        ops[9 + 4] = C(-1.0);     // sz (1,1)
        ops[18 + 2 + 3 * 1] = C(1.0);   // |r><1|: (2, 1)
        CUDA_OK(cudaMemcpy(E.nops, n, sizeof(n), cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(E.dops, ops, sizeof(ops), cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(E.d_sites, &a, sizeof(int), cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(E.d_driven, &a, sizeof(int), cudaMemcpyHostToDevice));
    }
}

// candidate rows (a + da*b), ordered by (a + b, a), for QR of node k w.r.t. leg o
void build_candidates(ttn_ctx* c) {
    for (int k = 0; k < (int)c->nodes.size(); ++k) {
        const Node& nd = c->nodes[k];
        for (int o = 0; o < 3; ++o) {
            int la = (o == 0) ? 1 : 0, lb = (o == 2) ? 1 : 2;
            int da = nd.d[la], db = nd.d[lb];
            auto allowed = [&](int leg, int idx) {
                if (leg == 2) return true;
                int ch = nd.child[leg];
                if (ch >= 0) return true;
                return c->leaf_atom[-ch - 1] >= 0 || idx == 0;
            };
            std::vector<std::pair<std::pair<int, int>, int>> rows;
            for (int b = 0; b < db; ++b)
                for (int a = 0; a < da; ++a)
                    if (allowed(la, a) && allowed(lb, b)) rows.push_back({{a + b, a}, a + da * b});
            std::sort(rows.begin(), rows.end());
            std::vector<int> h(rows.size());
            for (size_t i = 0; i < rows.size(); ++i) h[i] = rows[i].second;
            int* d = (int*)dalloc(c, sizeof(int) * std::max<size_t>(1, h.size()));
            if (!h.empty()) CUDA_OK(cudaMemcpy(d, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice));
            c->cand[{k, o}] = d;
            c->ncand[{k, o}] = (int)h.size();
        }
    }
}

void build_tree(ttn_ctx* c) {
    int side = 1;
    while (side < std::max(c->Lx, c->Ly)) side *= 2;
    c->leaf_atom.clear();
    for (int d = 0; d < side * side; ++d) {
        int x, y;
        hilbert_cell(side, d, x, y);
        if (x < c->Lx && y < c->Ly) c->leaf_atom.push_back(x + c->Lx * y);
    }
    int nl = 2;
    while (nl < (int)c->leaf_atom.size()) nl *= 2;
    c->leaf_atom.resize(nl, -1);
    c->n_leaves = nl;
    c->nodes.clear();
    c->level_nodes.clear();
    std::vector<int> cur;
    for (int i = 0; i < nl / 2; ++i) {
        Node nd;
        nd.child[0] = -(2 * i) - 1;
        nd.child[1] = -(2 * i + 1) - 1;
        nd.level = 0;
        for (int l = 2 * i; l <= 2 * i + 1; ++l)
            if (c->leaf_atom[l] >= 0) nd.sites.push_back(c->leaf_atom[l]);
        cur.push_back((int)c->nodes.size());
        c->nodes.push_back(nd);
    }
    c->level_nodes.push_back(cur);
    int lev = 0;
    while (cur.size() > 1) {
        ++lev;
        std::vector<int> nxt;
        for (size_t i = 0; i < cur.size() / 2; ++i) {
            Node nd;
            nd.child[0] = cur[2 * i];
            nd.child[1] = cur[2 * i + 1];
            nd.level = lev;
            int id = (int)c->nodes.size();
            for (int u = 0; u < 2; ++u) {
                c->nodes[nd.child[u]].parent = id;
                const auto& cs = c->nodes[nd.child[u]].sites;
                nd.sites.insert(nd.sites.end(), cs.begin(), cs.end());
            }
            nxt.push_back(id);
            c->nodes.push_back(nd);
        }
        cur = nxt;
        c->level_nodes.push_back(cur);
    }
    c->root = cur[0];
    // bond dims
    std::vector<int> pdim(c->nodes.size(), 1);
    for (int k = 0; k < (int)c->nodes.size(); ++k) {
        if (k == c->root) continue;
        int a = (int)c->nodes[k].sites.size();
        long long cap = c->chi + 1;
        pdim[k] = (int)std::min<long long>(c->chi, std::min(ipow3_capped(a, cap), ipow3_capped(c->N - a, cap)));
    }
    c->smax = 1;
    for (int k = 0; k < (int)c->nodes.size(); ++k) {
        Node& nd = c->nodes[k];
        for (int u = 0; u < 2; ++u) nd.d[u] = nd.child[u] >= 0 ? pdim[nd.child[u]] : 3;
        nd.d[2] = pdim[k];
        nd.s = (long long)nd.d[0] * nd.d[1] * nd.d[2];
        c->smax = std::max(c->smax, nd.s);
    }
}

// QR scratch for matrices of up to maxM rows and maxD columns.
void alloc_qr_scratch(ttn_ctx* c, long long maxM, int maxD, QrScratch& q) {
    const long long gq = (maxM + QR_ROWS - 1) / QR_ROWS;   // row blocks
    q.part = (cplx*)dalloc(c, sizeof(cplx) * 2 * gq * (2 * MAX_CHI + 4));   // two buffers of partial rows
    q.h = (cplx*)dalloc(c, sizeof(cplx) * 2 * (MAX_CHI + 2));   // two coefficient vectors
    q.pnorm = (double*)dalloc(c, sizeof(double) * std::max<long long>(gq, QR_FROB_BLOCKS));
    q.scal = (double*)dalloc(c, sizeof(double) * 8);
    q.flags = (int*)dalloc(c, sizeof(int) * (maxD + 2));
    q.rownorm = (double*)dalloc(c, sizeof(double) * std::max<long long>(maxM, 1));
    q.pick = (int*)dalloc(c, sizeof(int) * 4);
    q.kept = (int*)dalloc(c, sizeof(int) * (maxD + 2));
    q.dep = (int*)dalloc(c, sizeof(int) * (maxD + 2));
    q.acc_rows = (int*)dalloc(c, sizeof(int) * (maxD + 2));
    q.Y = (cplx*)dalloc(c, sizeof(cplx) * QR_SC_MAXR * (maxD + 2));
    q.nu = (double*)dalloc(c, sizeof(double) * (maxD + 2));
    q.row_rank = (int*)dalloc(c, sizeof(int) * std::max<long long>(maxM, 1));
    q.cand_used = (int*)dalloc(c, sizeof(int) * std::max<long long>(maxM, 1));
    q.bar = (unsigned*)dalloc(c, sizeof(unsigned) * 4);
    q.err = (int*)dalloc(c, sizeof(int) * 4);
    CUDA_OK(cudaMemset(q.err, 0, sizeof(int) * 4));
    CUDA_OK(cudaMemset(q.bar, 0, sizeof(unsigned) * 4));
}

void allocate(ttn_ctx* c) {
    int nn = (int)c->nodes.size();
    c->T.assign(nn, nullptr);
    for (int k = 0; k < nn; ++k) c->T[k] = (cplx*)dalloc(c, sizeof(cplx) * c->smax);
    for (int i = 0; i < 3; ++i) c->tmp[i] = (cplx*)dalloc(c, sizeof(cplx) * c->smax);
    // channel scratch: max over nodes of r * s, at least 8 * smax for op stacks
    long long zc = 8 * c->smax;
    long long gc = 1;
    for (int k = 0; k < nn; ++k) {
        const Node& nd = c->nodes[k];
        long long tot = c->N;
        long long in0 = (nd.child[0] >= 0) ? (long long)c->nodes[nd.child[0]].sites.size() : 1;
        long long in1 = (nd.child[1] >= 0) ? (long long)c->nodes[nd.child[1]].sites.size() : 1;
        long long out = tot - (long long)nd.sites.size();
        long long r = std::max({std::min(in0, in1), std::min(in0, out), std::min(in1, out)});
        zc = std::max(zc, r * nd.s);
        int Dm = std::max({nd.d[0], nd.d[1], nd.d[2]});
        gc = std::max(gc, std::max(r, (long long)c->N) * (long long)Dm * Dm);
    }
    c->zcap = zc;
    c->Z = (cplx*)dalloc(c, sizeof(cplx) * zc);
    c->gcap = gc;
    for (int i = 0; i < 3; ++i) c->Gbuf[i] = (cplx*)dalloc(c, sizeof(cplx) * gc);
    for (int i = 0; i < 3; ++i) c->hb[i] = (cplx*)dalloc(c, sizeof(cplx) * MAX_CHI * MAX_CHI);
    c->Rbuf = (cplx*)dalloc(c, sizeof(cplx) * MAX_CHI * MAX_CHI);
    c->dense_H = (cplx*)dalloc(c, sizeof(cplx) * SMALL_S * SMALL_S);
    c->Kbasis = (cplx*)dalloc(c, sizeof(cplx) * (KRYLOV_MMAX + 1) * c->smax);
    c->ks = (KrylovScalars*)dalloc(c, sizeof(KrylovScalars));
    c->kh1 = (cplx*)dalloc(c, sizeof(cplx) * (KRYLOV_MMAX + 1));
    c->kh2 = (cplx*)dalloc(c, sizeof(cplx) * (KRYLOV_MMAX + 1));
    c->kpart = (cplx*)dalloc(c, sizeof(cplx) * 2 * RED_BLOCKS * (MAX_CHI + 2));
    c->kpn = (double*)dalloc(c, sizeof(double) * RED_BLOCKS);
    c->apx = (double*)dalloc(c, sizeof(double) * RED_BLOCKS);
    c->apr = (double*)dalloc(c, sizeof(double) * RED_BLOCKS);
    long long mq = 1;   // largest QR row count: max over nodes and legs of s / d_leg
    for (int k = 0; k < nn; ++k)
        for (int u = 0; u < 3; ++u) mq = std::max(mq, c->nodes[k].s / c->nodes[k].d[u]);
    alloc_qr_scratch(c, mq, MAX_CHI, c->qr);
    c->d_coef = (double*)dalloc(c, sizeof(double) * 5 * c->N);
    c->h_coef.assign(5 * c->N, 0.0);
    CUDA_OK(cudaMallocHost(&c->hflag, 4 * sizeof(int)));
    c->up.assign(nn, Env());
    c->down.assign(nn, Env());
    c->phys.assign(c->n_leaves, Env());
    c->dummy = Env();
    c->dummy.D = 1;
    for (int k = 0; k < nn; ++k) {
        c->up[k].D = c->nodes[k].d[2];
        c->down[k].D = c->nodes[k].d[2];
    }
}

// Build node tensors from per-leaf branch vectors (3 x nb, column-major) and
// the root combination: every node is the QR-completed isometry of its
// branch columns (the same completion rule as the sweep's QR).
void build_from_branches(ttn_ctx* c, const std::vector<std::vector<zc>>& leaf_br, int nb,
                         const std::vector<zc>& root_coef) {
    int nn = (int)c->nodes.size();
    std::vector<std::vector<zc>> B(nn);   // per node: d2 x nb branch coordinates
    for (auto& lev : c->level_nodes) {
        for (int k : lev) {
            const Node& nd = c->nodes[k];
            const std::vector<zc>* col[2];
            int dd[2] = {nd.d[0], nd.d[1]};
            for (int u = 0; u < 2; ++u) {
                int ch = nd.child[u];
                col[u] = ch >= 0 ? &B[ch] : &leaf_br[-ch - 1];
            }
            long long M = (long long)dd[0] * dd[1];
            int D = nd.d[2];
            std::vector<zc> A(M * std::max(D, nb), zc(0.0));
            std::vector<zc> full(M * nb);
            for (int b = 0; b < nb; ++b)
                for (int j = 0; j < dd[1]; ++j)
                    for (int i = 0; i < dd[0]; ++i)
                        full[i + dd[0] * j + M * b] = (*col[0])[i + dd[0] * b] * (*col[1])[j + dd[1] * b];
            if (k == c->root) {
                std::vector<zc> X(M, zc(0.0));
                for (int b = 0; b < nb; ++b)
                    for (long long e = 0; e < M; ++e) X[e] += full[e + M * b] * root_coef[b];
                CUDA_OK(cudaMemcpy(c->T[k], X.data(), sizeof(cplx) * M, cudaMemcpyHostToDevice));
                continue;
            }
            int nk = std::min(nb, D);
            std::fill(A.begin(), A.end(), zc(0.0));
            for (long long e = 0; e < M * nk; ++e) A[e] = full[e];
            CUDA_OK(cudaMemcpy(c->T[k], A.data(), sizeof(cplx) * M * D, cudaMemcpyHostToDevice));
            int ndep = 0;
            auto key = std::make_pair(k, 2);
            if (qr_cgs2(c->T[k], (int)M, D, c->Rbuf, c->cand[key], c->ncand[key], c->qr, c->stream, &ndep) < 0)
                throw TtnError(TTN_ERR_TIMEOUT, "QR grid barrier wait timed out");
            std::vector<zc> R((size_t)D * D), Q(M * D);
            CUDA_OK(cudaMemcpyAsync(R.data(), c->Rbuf, sizeof(cplx) * D * D, cudaMemcpyDeviceToHost, c->stream));
            CUDA_OK(cudaMemcpyAsync(Q.data(), c->T[k], sizeof(cplx) * M * D, cudaMemcpyDeviceToHost, c->stream));
            CUDA_OK(cudaStreamSynchronize(c->stream));
            std::vector<zc> Bk((size_t)D * nb, zc(0.0));
            if (nb <= D) {
                for (int b = 0; b < nb; ++b)
                    for (int r = 0; r < D; ++r) Bk[r + D * b] = R[r + D * b];
            } else {
                for (int b = 0; b < nb; ++b)
                    for (int r = 0; r < D; ++r) {
                        zc s(0.0);
                        for (long long e = 0; e < M; ++e) s += std::conj(Q[e + M * r]) * full[e + M * b];
                        Bk[r + D * b] = s;
                    }
            }
            B[k] = Bk;
        }
    }
    c->centre = c->root;
    rebuild_up_envs(c);
}

void set_driven(ttn_ctx* c) {
    c->driven.assign(c->N, 0);
    for (const ttn_pulse& p : c->schedule)
        if (p.omega_x != 0.0 || p.omega_z != 0.0 || p.omega_r != 0.0) c->driven[p.atom] = 1;
}

void set_V(ttn_ctx* c) {
    int N = c->N;
    c->V.assign((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (i == j) continue;
            double dx = c->xy[2 * i] - c->xy[2 * j], dy = c->xy[2 * i + 1] - c->xy[2 * j + 1];
            double d = std::hypot(dx, dy);
            if (c->r_cut > 0 && d > c->r_cut) continue;
            c->V[(size_t)i * N + j] = c->C6 / std::pow(d, 6);
        }
    c->vsub.clear();   // device buffers stay owned by allocs
}

// ------------------------------------------------------------- observables
// <psi| op_i |psi> for ops renormalised to the root legs (centre at root).
void root_expect(ttn_ctx* c, const cplx* st0, int n0, const cplx* st1, int n1, std::vector<zc>& out) {
    ForceFp64 f64;
    const Node& nd = c->nodes[c->root];
    long long s = nd.s;
    out.assign(n0 + n1, zc(0.0));
    cplx* res = c->Gbuf[2];
    const cplx* st[2] = {st0, st1};
    int ns[2] = {n0, n1};
    int off = 0;
    for (int u = 0; u < 2; ++u) {
        if (ns[u] == 0) continue;
        long long DD = (long long)nd.d[u] * nd.d[u];
        int chunk = (int)std::max<long long>(1, c->zcap / s);
        for (int i0 = 0; i0 < ns[u]; i0 += chunk) {
            int nb = std::min(chunk, ns[u] - i0);
            leg_apply(c, st[u] + i0 * DD, nd.d[u], c->T[c->root], nd.d, u, c->Z, 0.0, nb, DD, s);
            project(c, c->T[c->root], nd.d, c->Z, nd.d, 2, res + off + i0, nb, s, 1);
        }
        off += ns[u];
    }
    std::vector<cplx> h(n0 + n1);
    CUDA_OK(cudaMemcpyAsync(h.data(), res, sizeof(cplx) * (n0 + n1), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n0 + n1; ++i) out[i] = zc(h[i].x, h[i].y);
}

double root_norm(ttn_ctx* c) {
    ForceFp64 f64;
    const Node& nd = c->nodes[c->root];
    project(c, c->T[c->root], nd.d, c->T[c->root], nd.d, 2, c->Gbuf[2], 1, 0, 0);
    cplx h;
    CUDA_OK(cudaMemcpyAsync(&h, c->Gbuf[2], sizeof(cplx), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    return h.x;
}

// Renormalise one diagonal one-site operator (per atom) up to the root legs.
void measure_projector(ttn_ctx* c, int level_index, std::vector<double>& out) {
    ForceFp64 f64;
    // bare operator: |level><level|
    cplx bare[9];
    for (int i = 0; i < 9; ++i) bare[i] = C(0.0);
    bare[level_index * 4] = C(1.0);
    int nn = (int)c->nodes.size();
    std::vector<cplx*> stack(nn, nullptr);
    std::vector<std::vector<int>> sites(nn);
    cplx* dbare = c->Gbuf[1];
    CUDA_OK(cudaMemcpyAsync(dbare, bare, sizeof(bare), cudaMemcpyHostToDevice, c->stream));
    std::vector<void*> temp;
    for (auto& lev : c->level_nodes)
        for (int k : lev) {
            if (k == c->root) continue;
            const Node& nd = c->nodes[k];
            long long DDo = (long long)nd.d[2] * nd.d[2];
            cplx* st = nullptr;
            CUDA_OK(cudaMalloc(&st, sizeof(cplx) * DDo * std::max<size_t>(1, nd.sites.size())));
            temp.push_back(st);
            long long off = 0;
            for (int u = 0; u < 2; ++u) {
                int ch = nd.child[u];
                if (ch < 0) {
                    if (c->leaf_atom[-ch - 1] < 0) continue;
                    renorm_stack(c, c->T[k], nd.d, u, 2, dbare, 1, st + off * DDo);
                    sites[k].push_back(c->leaf_atom[-ch - 1]);
                    off += 1;
                } else {
                    int n = (int)sites[ch].size();
                    renorm_stack(c, c->T[k], nd.d, u, 2, stack[ch], n, st + off * DDo);
                    sites[k].insert(sites[k].end(), sites[ch].begin(), sites[ch].end());
                    off += n;
                }
            }
            stack[k] = st;
        }
    const Node& rn = c->nodes[c->root];
    const cplx* st[2];
    int ns[2];
    std::vector<int> order;
    std::vector<cplx*> extra;
    for (int u = 0; u < 2; ++u) {
        int ch = rn.child[u];
        if (ch >= 0) {
            st[u] = stack[ch];
            ns[u] = (int)sites[ch].size();
            order.insert(order.end(), sites[ch].begin(), sites[ch].end());
        } else {
            int a = c->leaf_atom[-ch - 1];
            st[u] = dbare;
            ns[u] = a >= 0 ? 1 : 0;
            if (a >= 0) order.push_back(a);
        }
    }
    std::vector<zc> vals;
    root_expect(c, st[0], ns[0], st[1], ns[1], vals);
    out.assign(c->N, 0.0);
    for (size_t i = 0; i < order.size(); ++i) out[order[i]] = vals[i].real();
    for (void* p : temp) cudaFree(p);
}

zc overlap(ttn_ctx* psi, const ttn_ctx* tgt) {
    ForceFp64 f64;
    ttn_ctx* c = psi;
    int nn = (int)c->nodes.size();
    std::vector<cplx*> M(nn, nullptr);
    std::vector<void*> temp;
    for (auto& lev : c->level_nodes)
        for (int k : lev) {
            const Node& nd = c->nodes[k];
            const Node& nt = tgt->nodes[k];
            // W = M_c0 x_0 psi_k, then M_c1 x_1 W
            const cplx* cur = c->T[k];
            int d[3] = {nd.d[0], nd.d[1], nd.d[2]};
            cplx* bufs[2] = {c->tmp[0], c->tmp[1]};
            int bi = 0;
            for (int u = 0; u < 2; ++u) {
                int ch = nd.child[u];
                if (ch < 0) continue;
                leg_apply(c, M[ch], nt.d[u], cur, d, u, bufs[bi], 0.0);
                d[u] = nt.d[u];
                cur = bufs[bi];
                bi ^= 1;
            }
            cplx* out = nullptr;
            CUDA_OK(cudaMalloc(&out, sizeof(cplx) * (size_t)nt.d[2] * nd.d[2]));
            temp.push_back(out);
            project(c, tgt->T[k], nt.d, cur, d, 2, out, 1, 0, 0);
            M[k] = out;
        }
    cplx h;
    CUDA_OK(cudaMemcpyAsync(&h, M[c->root], sizeof(cplx), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    for (void* p : temp) cudaFree(p);
    return zc(h.x, h.y);
}

double energy(ttn_ctx* c) {
    ForceFp64 f64;
    compute_coef(c, c->t);
    int k = c->root;
    const Node& nd = c->nodes[k];
    const Env* e[3] = {&env_of(c, k, 0), &env_of(c, k, 1), &env_of(c, k, 2)};
    cplx* hbs[3] = {nullptr, nullptr, nullptr};
    int Dl[3] = {nd.d[0], nd.d[1], nd.d[2]};
    for (int u = 0; u < 3; ++u)
        if (env_has_block(*e[u])) {
            assemble(c, *e[u], c->hb[u]);
            hbs[u] = c->hb[u];
        }
    Pair pairs[3];
    int np = setup_pairs(c, e, pairs);
    heff_apply(c, nd.d, hbs, Dl, pairs, np, c->T[k], c->tmp[2]);
    project(c, c->T[k], nd.d, c->tmp[2], nd.d, 2, c->Gbuf[2], 1, 0, 0);
    cplx h;
    CUDA_OK(cudaMemcpyAsync(&h, c->Gbuf[2], sizeof(cplx), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    return h.x;
}

void sync_check(ttn_ctx* c) {
    CUDA_OK(cudaStreamSynchronize(c->stream));
    CUDA_OK(cudaGetLastError());
    check_split_flag(c);
}

template <class F>
ttn_status guard(ttn_ctx* c, F f) {
    try {
        f();
        return TTN_OK;
    } catch (const TtnError& e) {
        if (c) c->err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        if (c) c->err = e.what();
        return TTN_ERR_ALLOC;
    }
}

}  // namespace

// =================================================================== C ABI
extern "C" {

ttn_status ttn_create(int Lx, int Ly, int levels, int chi, ttn_ctx** out) {
    if (!out) return TTN_ERR_ARG;
    *out = nullptr;
    if (levels != 3 || chi < 1 || chi > MAX_CHI || Lx < 1 || Ly < 1 || (long long)Lx * Ly > MAX_ATOMS)
        return TTN_ERR_ARG;
    ttn_ctx* c = new ttn_ctx();
    c->Lx = Lx;
    c->Ly = Ly;
    c->N = Lx * Ly;
    c->chi = chi;
    ttn_status st = guard(c, [&] {
        build_tree(c);
        allocate(c);
        build_candidates(c);
        c->xy.resize(2 * c->N);
        for (int i = 0; i < c->N; ++i) {
            c->xy[2 * i] = i % Lx;
            c->xy[2 * i + 1] = i / Lx;
        }
        c->C6 = 0.0;
        set_V(c);
        c->driven.assign(c->N, 0);
        set_phys_envs(c);
        std::vector<std::vector<zc>> lb(c->n_leaves, std::vector<zc>{1.0, 0.0, 0.0});
        build_from_branches(c, lb, 1, {zc(1.0)});
        sync_check(c);
    });
    if (st != TTN_OK) {
        fprintf(stderr, "ttn_create: %s\n", c->err.c_str());
        ttn_destroy(c);
        return st;
    }
    *out = c;
    return TTN_OK;
}

void ttn_destroy(ttn_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (void* p : c->allocs) cudaFree(p);
    if (c->split_ws) cudaFree(c->split_ws);
    if (c->f64_ws) cudaFree(c->f64_ws);
    for (int i = 0; i < 3; ++i) {
        if (c->shP[i]) cudaFree(c->shP[i]);
        if (c->shQ[i]) cudaFree(c->shQ[i]);
        if (c->shG[i]) cudaFree(c->shG[i]);
        if (c->shX[i]) cudaFree(c->shX[i]);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->hflag) cudaFreeHost(c->hflag);
    delete c;
}

const char* ttn_last_error(const ttn_ctx* c) { return c ? c->err.c_str() : "null context"; }

ttn_status ttn_set_stream(ttn_ctx* c, void* s) {
    if (!c) return TTN_ERR_ARG;
    c->stream = (cudaStream_t)s;
    return TTN_OK;
}

ttn_status ttn_set_precision(ttn_ctx* c, ttn_precision p) {
    if (!c || (p != TTN_FP64 && p != TTN_SPLIT_TF32X3)) return TTN_ERR_ARG;
    c->prec = p;
    return TTN_OK;
}

ttn_status ttn_set_hamiltonian(ttn_ctx* c, const double* xy, double C6, double r_cut) {
    if (!c || !xy || !std::isfinite(C6) || !std::isfinite(r_cut)) return TTN_ERR_ARG;
    for (int i = 0; i < 2 * c->N; ++i)
        if (!std::isfinite(xy[i])) return TTN_ERR_ARG;
    for (int i = 0; i < c->N; ++i)
        for (int j = i + 1; j < c->N; ++j)
            if (xy[2 * i] == xy[2 * j] && xy[2 * i + 1] == xy[2 * j + 1]) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        c->xy.assign(xy, xy + 2 * c->N);
        c->C6 = C6;
        c->r_cut = r_cut;
        set_V(c);
        rebuild_up_envs(c);
        sync_check(c);
    });
}

ttn_status ttn_set_decay(ttn_ctx* c, double gamma) {
    if (!c || !std::isfinite(gamma) || gamma < 0.0) return TTN_ERR_ARG;
    c->gamma = gamma;
    return TTN_OK;
}

ttn_status ttn_apply_pulse(ttn_ctx* c, const ttn_pulse* sched, int n) {
    if (!c || n < 0 || (n > 0 && !sched)) return TTN_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const ttn_pulse& p = sched[i];
        if (p.atom < 0 || p.atom >= c->N || !(p.t1 >= p.t0) || !std::isfinite(p.omega_x) ||
            !std::isfinite(p.omega_z) || !std::isfinite(p.omega_r) || !std::isfinite(p.phase_r) ||
            !std::isfinite(p.delta))
            return TTN_ERR_ARG;
    }
    return guard(c, [&] {
        std::vector<int> old = c->driven;
        c->schedule.assign(sched, sched + n);
        set_driven(c);
        if (old != c->driven) {
            centre_to_root(c);
            set_phys_envs(c);
            rebuild_up_envs(c);
        }
        sync_check(c);
    });
}

ttn_status ttn_set_product_state(ttn_ctx* c, const double* amps) {
    if (!c || !amps) return TTN_ERR_ARG;
    for (int i = 0; i < 6 * c->N; ++i)
        if (!std::isfinite(amps[i])) return TTN_ERR_ARG;
    return guard(c, [&] {
        std::vector<std::vector<zc>> lb(c->n_leaves);
        for (int l = 0; l < c->n_leaves; ++l) {
            int a = c->leaf_atom[l];
            if (a < 0) lb[l] = {1.0, 0.0, 0.0};
            else lb[l] = {zc(amps[6 * a], amps[6 * a + 1]), zc(amps[6 * a + 2], amps[6 * a + 3]),
                          zc(amps[6 * a + 4], amps[6 * a + 5])};
        }
        build_from_branches(c, lb, 1, {zc(1.0)});
        c->t = 0.0;
        sync_check(c);
    });
}

ttn_status ttn_set_ghz_target(ttn_ctx* c, const int* mask, double phase) {
    if (!c || !mask || !std::isfinite(phase)) return TTN_ERR_ARG;
    return guard(c, [&] {
        std::vector<std::vector<zc>> lb(c->n_leaves);
        for (int l = 0; l < c->n_leaves; ++l) {
            int a = c->leaf_atom[l];
            // column-major 3 x 2: branch 0 = |0>, branch 1 = |1> on mask atoms
            std::vector<zc> m(6, zc(0.0));
            m[0] = 1.0;
            if (a >= 0 && mask[a]) m[3 + 1] = 1.0;
            else m[3 + 0] = 1.0;
            lb[l] = m;
        }
        double r = 1.0 / std::sqrt(2.0);
        build_from_branches(c, lb, 2, {zc(r), std::polar(r, phase)});
        sync_check(c);
    });
}

ttn_status ttn_tdvp_step(ttn_ctx* c, double dt) {
    if (!c || !(dt > 0.0) || !std::isfinite(dt)) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        compute_coef(c, c->t + 0.5 * dt);
        sweep_fwd(c, c->root, 0.5 * dt);
        sweep_rev(c, c->root, 0.5 * dt);
        c->t += dt;
        sync_check(c);
    });
}

ttn_status ttn_overlap(ttn_ctx* c, const ttn_ctx* tgt, double* re_im) {
    if (!c || !tgt || !re_im || tgt->Lx != c->Lx || tgt->Ly != c->Ly) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        if (tgt->centre != tgt->root) throw TtnError(TTN_ERR_STATE, "target centre is not at its root");
        if (tgt->stream != c->stream) CUDA_OK(cudaStreamSynchronize(tgt->stream));
        zc o = overlap(c, tgt);
        re_im[0] = o.real();
        re_im[1] = o.imag();
    });
}

ttn_status ttn_fidelity(ttn_ctx* c, const ttn_ctx* tgt, double* F) {
    if (!F) return TTN_ERR_ARG;
    double o[2];
    ttn_status st = ttn_overlap(c, tgt, o);
    if (st == TTN_OK) *F = o[0] * o[0] + o[1] * o[1];
    return st;
}

ttn_status ttn_measure(ttn_ctx* c, int which, double* out) {
    if (!c || !out || which < 0 || which > 2) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        std::vector<double> v;
        if (which == 2) {
            // n stacks are kept in the environments of the root's children
            const Env& e0 = env_of(c, c->root, 0);
            const Env& e1 = env_of(c, c->root, 1);
            std::vector<zc> vals;
            root_expect(c, e0.nops, (int)e0.sites.size(), e1.nops, (int)e1.sites.size(), vals);
            v.assign(c->N, 0.0);
            size_t i = 0;
            for (int a : e0.sites) v[a] = vals[i++].real();
            for (int a : e1.sites) v[a] = vals[i++].real();
        } else {
            measure_projector(c, which, v);
        }
        std::copy(v.begin(), v.end(), out);
    });
}

ttn_status ttn_norm(ttn_ctx* c, double* out) {
    if (!c || !out) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        *out = root_norm(c);
    });
}

ttn_status ttn_energy(ttn_ctx* c, double* out) {
    if (!c || !out) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        *out = energy(c);
    });
}

ttn_status ttn_get_time(ttn_ctx* c, double* t) {
    if (!c || !t) return TTN_ERR_ARG;
    *t = c->t;
    return TTN_OK;
}

ttn_status ttn_get_dense(ttn_ctx* c, double* psi) {
    if (!c || !psi || c->N > 9) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        sync_check(c);
        int nn = (int)c->nodes.size();
        // per node: vector over its leaves (leaf order, first fastest) x D
        std::vector<std::vector<zc>> vec(nn);
        std::vector<std::vector<int>> leaves(nn);
        for (auto& lev : c->level_nodes)
            for (int k : lev) {
                const Node& nd = c->nodes[k];
                std::vector<zc> X(nd.s);
                CUDA_OK(cudaMemcpy(X.data(), c->T[k], sizeof(cplx) * nd.s, cudaMemcpyDeviceToHost));
                std::vector<zc> part[2];
                long long dimL[2];
                for (int u = 0; u < 2; ++u) {
                    int ch = nd.child[u];
                    if (ch < 0) {
                        part[u].assign(9, zc(0.0));
                        for (int i = 0; i < 3; ++i) part[u][i + 3 * i] = 1.0;
                        dimL[u] = 3;
                        leaves[k].push_back(-ch - 1);
                    } else {
                        part[u] = vec[ch];
                        dimL[u] = (long long)part[u].size() / nd.d[u];
                        leaves[k].insert(leaves[k].end(), leaves[ch].begin(), leaves[ch].end());
                    }
                }
                long long L0 = dimL[0], L1 = dimL[1];
                int D = nd.d[2];
                std::vector<zc> out(L0 * L1 * D, zc(0.0));
                for (int cc = 0; cc < D; ++cc)
                    for (int b = 0; b < nd.d[1]; ++b)
                        for (int a = 0; a < nd.d[0]; ++a) {
                            zc x = X[a + nd.d[0] * (b + (long long)nd.d[1] * cc)];
                            if (x == zc(0.0)) continue;
                            for (long long j = 0; j < L1; ++j) {
                                zc y = x * part[1][j + L1 * b];
                                if (y == zc(0.0)) continue;
                                for (long long i = 0; i < L0; ++i)
                                    out[i + L0 * (j + L1 * cc)] += part[0][i + L0 * a] * y;
                            }
                        }
                vec[k] = out;
            }
        const std::vector<zc>& R = vec[c->root];
        const std::vector<int>& lv = leaves[c->root];
        long long dim = 1;
        for (int i = 0; i < c->N; ++i) dim *= 3;
        std::fill(psi, psi + 2 * dim, 0.0);
        long long total = (long long)R.size();
        for (long long e = 0; e < total; ++e) {
            long long r = e, idx = 0;
            bool ok = true;
            for (size_t q = 0; q < lv.size(); ++q) {
                int lvl = (int)(r % 3);
                r /= 3;
                int a = c->leaf_atom[lv[q]];
                if (a < 0) {
                    if (lvl != 0) ok = false;
                    continue;
                }
                long long p3 = 1;
                for (int i = 0; i < a; ++i) p3 *= 3;
                idx += lvl * p3;
            }
            if (!ok) continue;
            psi[2 * idx] += R[e].real();
            psi[2 * idx + 1] += R[e].imag();
        }
    });
}

ttn_status ttn_save(ttn_ctx* c, const char* path) {
    if (!c || !path) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        sync_check(c);
        FILE* f = fopen(path, "wb");
        if (!f) throw TtnError(TTN_ERR_ARG, "cannot open file");
        int hdr[4] = {c->Lx, c->Ly, c->chi, (int)c->nodes.size()};
        fwrite("TTN1", 1, 4, f);
        fwrite(hdr, sizeof(int), 4, f);
        fwrite(&c->t, sizeof(double), 1, f);
        for (int k = 0; k < (int)c->nodes.size(); ++k) {
            std::vector<cplx> X(c->nodes[k].s);
            CUDA_OK(cudaMemcpy(X.data(), c->T[k], sizeof(cplx) * X.size(), cudaMemcpyDeviceToHost));
            fwrite(X.data(), sizeof(cplx), X.size(), f);
        }
        fclose(f);
    });
}

ttn_status ttn_load(ttn_ctx* c, const char* path) {
    if (!c || !path) return TTN_ERR_ARG;
    return guard(c, [&] {
        FILE* f = fopen(path, "rb");
        if (!f) throw TtnError(TTN_ERR_ARG, "cannot open file");
        char magic[4];
        int hdr[4];
        double t;
        bool ok = fread(magic, 1, 4, f) == 4 && std::memcmp(magic, "TTN1", 4) == 0 &&
                  fread(hdr, sizeof(int), 4, f) == 4 && fread(&t, sizeof(double), 1, f) == 1 &&
                  hdr[0] == c->Lx && hdr[1] == c->Ly && hdr[2] == c->chi && hdr[3] == (int)c->nodes.size();
        std::vector<std::vector<cplx>> data;
        for (int k = 0; ok && k < (int)c->nodes.size(); ++k) {
            std::vector<cplx> X(c->nodes[k].s);
            ok = fread(X.data(), sizeof(cplx), X.size(), f) == X.size();
            data.push_back(X);
        }
        fclose(f);
        if (!ok) throw TtnError(TTN_ERR_ARG, "file does not match this context");
        for (int k = 0; k < (int)c->nodes.size(); ++k)
            CUDA_OK(cudaMemcpy(c->T[k], data[k].data(), sizeof(cplx) * data[k].size(), cudaMemcpyHostToDevice));
        c->t = t;
        c->centre = c->root;
        rebuild_up_envs(c);
        sync_check(c);
    });
}

ttn_status ttn_num_nodes(const ttn_ctx* c, int* n) {
    if (!c || !n) return TTN_ERR_ARG;
    *n = (int)c->nodes.size();
    return TTN_OK;
}

ttn_status ttn_node_info(const ttn_ctx* c, int k, int* dims, int* children) {
    if (!c || k < 0 || k >= (int)c->nodes.size()) return TTN_ERR_ARG;
    for (int u = 0; u < 3; ++u)
        if (dims) dims[u] = c->nodes[k].d[u];
    for (int u = 0; u < 2; ++u)
        if (children) children[u] = c->nodes[k].child[u];
    return TTN_OK;
}

ttn_status ttn_leaf_atoms(const ttn_ctx* c, int* la, int* n) {
    if (!c || !n) return TTN_ERR_ARG;
    if (la) std::copy(c->leaf_atom.begin(), c->leaf_atom.end(), la);
    *n = c->n_leaves;
    return TTN_OK;
}

ttn_status ttn_get_node(ttn_ctx* c, int k, double* data) {
    if (!c || !data || k < 0 || k >= (int)c->nodes.size()) return TTN_ERR_ARG;
    return guard(c, [&] {
        CUDA_OK(cudaMemcpyAsync(data, c->T[k], sizeof(cplx) * c->nodes[k].s, cudaMemcpyDeviceToHost, c->stream));
        CUDA_OK(cudaStreamSynchronize(c->stream));
    });
}

ttn_status ttn_set_node(ttn_ctx* c, int k, const double* data) {
    if (!c || !data || k < 0 || k >= (int)c->nodes.size()) return TTN_ERR_ARG;
    return guard(c, [&] {
        CUDA_OK(cudaMemcpyAsync(c->T[k], data, sizeof(cplx) * c->nodes[k].s, cudaMemcpyHostToDevice, c->stream));
        CUDA_OK(cudaStreamSynchronize(c->stream));
        c->centre = c->root;
    });
}

ttn_status ttn_refresh_envs(ttn_ctx* c) {
    if (!c) return TTN_ERR_ARG;
    return guard(c, [&] {
        c->centre = c->root;
        rebuild_up_envs(c);
        sync_check(c);
    });
}

ttn_status ttn_apply_heff(ttn_ctx* c, int k, const double* x, double* y) {
    if (!c || !x || !y || k < 0 || k >= (int)c->nodes.size()) return TTN_ERR_ARG;
    return guard(c, [&] {
        centre_to_root(c);
        centre_to(c, k);
        compute_coef(c, c->t);
        const Node& nd = c->nodes[k];
        CUDA_OK(cudaMemcpyAsync(c->tmp[1], x, sizeof(cplx) * nd.s, cudaMemcpyHostToDevice, c->stream));
        const Env* e[3] = {&env_of(c, k, 0), &env_of(c, k, 1), &env_of(c, k, 2)};
        cplx* hbs[3] = {nullptr, nullptr, nullptr};
        int Dl[3] = {nd.d[0], nd.d[1], nd.d[2]};
        for (int u = 0; u < 3; ++u)
            if (env_has_block(*e[u])) {
                assemble(c, *e[u], c->hb[u]);
                hbs[u] = c->hb[u];
            }
        Pair pairs[3];
        int np = setup_pairs(c, e, pairs);
        SplitHeff S;
        if (split_heff_prepare(c, S, nd.d, hbs, pairs, np)) split_heff_apply(c, S, c->tmp[1], c->tmp[2]);
        else heff_apply(c, nd.d, hbs, Dl, pairs, np, c->tmp[1], c->tmp[2]);
        CUDA_OK(cudaMemcpyAsync(y, c->tmp[2], sizeof(cplx) * nd.s, cudaMemcpyDeviceToHost, c->stream));
        sync_check(c);
    });
}

ttn_status ttn_profile_begin(ttn_ctx* c) {
    if (!c) return TTN_ERR_ARG;
    return guard(c, [&] {
        CUDA_OK(cudaStreamSynchronize(c->stream));
        c->prof.clear();
        c->ev_next = 0;
        c->profiling = true;
    });
}

ttn_status ttn_profile_end(ttn_ctx* c, double* out, int n) {
    if (!c || !out || n < 16) return TTN_ERR_ARG;
    const int nk = std::min((int)PK_N, n / 4);   // kinds that fit in out
    return guard(c, [&] {
        c->profiling = false;
        CUDA_OK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < 4 * nk; ++i) out[i] = 0.0;
        c->prof_last.clear();
        for (auto& r : c->prof) {
            float ms = 0.f;
            CUDA_OK(cudaEventElapsedTime(&ms, r.e0, r.e1));
            c->prof_last.push_back({(double)r.kind, (double)r.shape[0], (double)r.shape[1], (double)r.shape[2],
                                    (double)r.shape[3], (double)ms, r.flops});
            if (r.kind >= nk) continue;
            out[4 * r.kind + 0] += 1.0;
            out[4 * r.kind + 1] += ms;
            out[4 * r.kind + 2] += r.flops;
            out[4 * r.kind + 3] += r.bytes;
        }
        c->prof.clear();
        c->ev_next = 0;
    });
}

// Random (seeded, uniform in [-1, 1)) complex operands, C = A B with A M x K
// and B K x N column-major, in FP64 and in the chosen precision.
__global__ void selftest_fill(cplx* x, long long n, unsigned long long seed, int tf32_exact) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(e + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        double re = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        z = z * 0x2545F4914F6CDD1DULL + 1;
        z ^= z >> 29;
        double im = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        if (tf32_exact) {   // keep 11 significant bits: exactly representable in TF32
            re = (double)__uint_as_float(__float_as_uint((float)re) & 0xFFFFE000u);
            im = (double)__uint_as_float(__float_as_uint((float)im) & 0xFFFFE000u);
        }
        x[e] = make_double2(re, im);
    }
}

ttn_status ttn_selftest_contract(int M, int N, int K, int precision, unsigned long long seed, int tf32_exact,
                                 double* rel_err) {
    if (M < 1 || N < 1 || K < 1 || !rel_err || (long long)M * N > (1LL << 26) || (long long)M * K > (1LL << 26) ||
        (long long)K * N > (1LL << 26))
        return TTN_ERR_ARG;
    ttn_ctx tmp;
    tmp.prec = (ttn_precision)precision;
    return guard(&tmp, [&] {
        cplx *A = (cplx*)dalloc(&tmp, sizeof(cplx) * M * K), *B = (cplx*)dalloc(&tmp, sizeof(cplx) * K * N);
        cplx *C0 = (cplx*)dalloc(&tmp, sizeof(cplx) * M * N), *C1 = (cplx*)dalloc(&tmp, sizeof(cplx) * M * N);
        selftest_fill<<<256, 256>>>(A, (long long)M * K, seed, tf32_exact);
        selftest_fill<<<256, 256>>>(B, (long long)K * N, seed * 31 + 7, tf32_exact);
        GemmArgs g = base_args();
        g.M = M; g.N = N; g.Ki = K;
        g.A = A; g.a_m = 1; g.a_ki = M;
        g.B = B; g.b_ki = 1; g.b_n = K;
        g.C = C0; g.c_m = 1; g.c_n = M;
        launch_zgemm_f64(g, nullptr);
        g.C = C1;
        tmp.stream = nullptr;
        gemm(&tmp, g);
        CUDA_OK(cudaDeviceSynchronize());
        std::vector<cplx> h0((size_t)M * N), h1((size_t)M * N);
        CUDA_OK(cudaMemcpy(h0.data(), C0, sizeof(cplx) * h0.size(), cudaMemcpyDeviceToHost));
        CUDA_OK(cudaMemcpy(h1.data(), C1, sizeof(cplx) * h1.size(), cudaMemcpyDeviceToHost));
        double mx = 0.0, me = 0.0;
        for (size_t i = 0; i < h0.size(); ++i) {
            mx = std::max(mx, std::hypot(h0[i].x, h0[i].y));
            me = std::max(me, std::hypot(h1[i].x - h0[i].x, h1[i].y - h0[i].y));
        }
        *rel_err = mx > 0 ? me / mx : me;
        for (void* p : tmp.allocs) cudaFree(p);
        tmp.allocs.clear();
        if (tmp.split_ws) cudaFree(tmp.split_ws);
        tmp.split_ws = nullptr;
        if (tmp.f64_ws) cudaFree(tmp.f64_ws);
        tmp.f64_ws = nullptr;
    });
}

ttn_status ttn_selftest_qr(const double* A, int M, int D, const int* cand, int ncand, double* Q, double* R,
                          int* n_dependent, float* ms) {
    if (M < 1 || D < 1 || D > MAX_CHI || M < D || (long long)M * D > (1LL << 26) || !A || !Q || !R ||
        (cand && (ncand < 1 || ncand > M)))
        return TTN_ERR_ARG;
    if (cand)
        for (int i = 0; i < ncand; ++i)
            if (cand[i] < 0 || cand[i] >= M) return TTN_ERR_ARG;
    ttn_ctx tmp;
    return guard(&tmp, [&] {
        struct Free {
            ttn_ctx* t;
            ~Free() {
                for (void* p : t->allocs) cudaFree(p);
                t->allocs.clear();
            }
        } fr{&tmp};
        QrScratch q;
        alloc_qr_scratch(&tmp, M, D, q);
        cplx* dA = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)M * D);
        cplx* dR = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)D * D);
        const int nc = cand ? ncand : M;
        int* dc = (int*)dalloc(&tmp, sizeof(int) * nc);
        std::vector<int> hc(nc);
        for (int i = 0; i < nc; ++i) hc[i] = cand ? cand[i] : i;
        CUDA_OK(cudaMemcpy(dc, hc.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(dA, A, sizeof(cplx) * (size_t)M * D, cudaMemcpyHostToDevice));
        cudaEvent_t e0, e1;
        CUDA_OK(cudaEventCreate(&e0));
        CUDA_OK(cudaEventCreate(&e1));
        int ndep = 0;
        CUDA_OK(cudaEventRecord(e0, nullptr));
        int nl = qr_cgs2(dA, M, D, dR, dc, nc, q, nullptr, &ndep);
        CUDA_OK(cudaEventRecord(e1, nullptr));
        CUDA_OK(cudaEventSynchronize(e1));
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (nl < 0) throw TtnError(TTN_ERR_TIMEOUT, "QR grid barrier wait timed out");
        CUDA_OK(cudaGetLastError());
        CUDA_OK(cudaMemcpy(Q, dA, sizeof(cplx) * (size_t)M * D, cudaMemcpyDeviceToHost));
        CUDA_OK(cudaMemcpy(R, dR, sizeof(cplx) * (size_t)D * D, cudaMemcpyDeviceToHost));
        if (n_dependent) *n_dependent = ndep;
        if (ms) *ms = t;
    });
}

ttn_status ttn_selftest_contract_host(const double* A, const double* B, double* Cout, int M, int N, int K,
                                      int precision, int* path, float* ms) {
    if (!A || !B || !Cout || M < 1 || N < 1 || K < 1 || (long long)M * N > (1LL << 26) ||
        (long long)M * K > (1LL << 26) || (long long)K * N > (1LL << 26) ||
        (precision != TTN_FP64 && precision != TTN_SPLIT_TF32X3))
        return TTN_ERR_ARG;
    ttn_ctx tmp;
    tmp.prec = (ttn_precision)precision;
    return guard(&tmp, [&] {
        struct Free {
            ttn_ctx* t;
            ~Free() {
                for (void* p : t->allocs) cudaFree(p);
                t->allocs.clear();
                if (t->split_ws) cudaFree(t->split_ws);
                t->split_ws = nullptr;
                if (t->f64_ws) cudaFree(t->f64_ws);
                t->f64_ws = nullptr;
            }
        } fr{&tmp};
        cplx* dA = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)M * K);
        cplx* dB = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)K * N);
        cplx* dC = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)M * N);
        CUDA_OK(cudaMemcpy(dA, A, sizeof(cplx) * (size_t)M * K, cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(dB, B, sizeof(cplx) * (size_t)K * N, cudaMemcpyHostToDevice));
        GemmArgs g = base_args();
        g.M = M; g.N = N; g.Ki = K;
        g.A = dA; g.a_m = 1; g.a_ki = M;
        g.B = dB; g.b_ki = 1; g.b_n = K;
        g.C = dC; g.c_m = 1; g.c_n = M;
        const bool tc = precision == TTN_SPLIT_TF32X3 && split_workspace_bytes(g) > 0;
        if (tc) grow_split_ws(&tmp, split_workspace_bytes(g));   // outside the timed region
        cudaEvent_t e0, e1;
        CUDA_OK(cudaEventCreate(&e0));
        CUDA_OK(cudaEventCreate(&e1));
        CUDA_OK(cudaEventRecord(e0, nullptr));
        gemm(&tmp, g);
        CUDA_OK(cudaEventRecord(e1, nullptr));
        CUDA_OK(cudaEventSynchronize(e1));
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CUDA_OK(cudaGetLastError());
        check_split_flag(&tmp);
        CUDA_OK(cudaMemcpy(Cout, dC, sizeof(cplx) * (size_t)M * N, cudaMemcpyDeviceToHost));
        if (path) *path = tc ? 1 : 0;
        if (ms) *ms = t;
    });
}

ttn_status ttn_selftest_fp64_peak(int method, double* tflops) {
    if (!tflops || (method != 0 && method != 1)) return TTN_ERR_ARG;
    ttn_ctx tmp;
    return guard(&tmp, [&] {
        struct Free {
            ttn_ctx* t;
            ~Free() {
                for (void* p : t->allocs) cudaFree(p);
                t->allocs.clear();
            }
        } fr{&tmp};
        double* out = (double*)dalloc(&tmp, 64);
        int dev = 0, nsm = 0;
        CUDA_OK(cudaGetDevice(&dev));
        CUDA_OK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int blocks = 8 * nsm;   // 2048 threads per SM: every FP64 unit busy
        cudaEvent_t e0, e1;
        CUDA_OK(cudaEventCreate(&e0));
        CUDA_OK(cudaEventCreate(&e1));
        k_fp64_probe(method, blocks, 64, out, nullptr);   // warm-up
        int iters = 256;
        float t = 0.f;
        double fl = 0.0;
        for (int rep = 0; rep < 12; ++rep) {   // grow until a launch takes >= 20 ms
            CUDA_OK(cudaEventRecord(e0, nullptr));
            fl = k_fp64_probe(method, blocks, iters, out, nullptr);
            CUDA_OK(cudaEventRecord(e1, nullptr));
            CUDA_OK(cudaEventSynchronize(e1));
            CUDA_OK(cudaGetLastError());
            cudaEventElapsedTime(&t, e0, e1);
            if (t >= 20.f) break;
            iters *= 2;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *tflops = fl / (t * 1e-3) / 1e12;
    });
}

ttn_status ttn_svd_truncate(const double* A, int M, int N, int chi, double eps, double* U, double* S, double* Vh,
                            int* k_out, double* discarded) {
    if (!A || !U || !S || !Vh || !k_out || M < 1 || N < 1 || N > MAX_CHI || M < N || chi < 1 || !(eps >= 0.0) ||
        (long long)M * N > (1LL << 26))
        return TTN_ERR_ARG;
    ttn_ctx tmp;
    return guard(&tmp, [&] {
        struct Free {
            ttn_ctx* t;
            ~Free() {
                for (void* p : t->allocs) cudaFree(p);
                t->allocs.clear();
            }
        } fr{&tmp};
        QrScratch q;
        alloc_qr_scratch(&tmp, M, N, q);
        cplx* dA = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)M * N);
        cplx* dR = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)N * N);
        cplx* dV = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)N * N);
        cplx* dUr = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)N * N);
        cplx* dVh = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)N * N);
        cplx* dU = (cplx*)dalloc(&tmp, sizeof(cplx) * (size_t)M * N);
        double* dS = (double*)dalloc(&tmp, sizeof(double) * N);
        int* dorder = (int*)dalloc(&tmp, sizeof(int) * N);
        int* dk = (int*)dalloc(&tmp, sizeof(int) * 4);
        double* ddisc = (double*)dalloc(&tmp, sizeof(double));
        unsigned* bar = (unsigned*)dalloc(&tmp, sizeof(unsigned) * 4);
        int* err = (int*)dalloc(&tmp, sizeof(int) * 4);
        int* info = (int*)dalloc(&tmp, sizeof(int) * 4);
        int* cand = (int*)dalloc(&tmp, sizeof(int) * M);
        std::vector<int> hc(M);
        for (int i = 0; i < M; ++i) hc[i] = i;
        CUDA_OK(cudaMemcpy(cand, hc.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemcpy(dA, A, sizeof(cplx) * (size_t)M * N, cudaMemcpyHostToDevice));
        CUDA_OK(cudaMemset(err, 0, sizeof(int) * 4));
        int ndep = 0;
        if (qr_cgs2(dA, M, N, dR, cand, M, q, nullptr, &ndep) < 0)
            throw TtnError(TTN_ERR_TIMEOUT, "QR grid barrier wait timed out");
        if (svd_jacobi_square(dR, dV, N, 60, 1e-15, bar, err, info, nullptr) < 0)
            throw TtnError(TTN_ERR_CUDA, "Jacobi SVD launch failed");
        int herr = 0;
        CUDA_OK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) throw TtnError(TTN_ERR_TIMEOUT, "Jacobi SVD grid barrier wait timed out");
        svd_finish(dR, dV, N, chi, eps, dUr, dVh, dS, dk, ddisc, dorder, nullptr);
        int k = 0;
        CUDA_OK(cudaMemcpy(&k, dk, sizeof(int), cudaMemcpyDeviceToHost));
        GemmArgs g = base_args();   // U = Q Ur
        g.M = M; g.N = k; g.Ki = N;
        g.A = dA; g.a_m = 1; g.a_ki = M;
        g.B = dUr; g.b_ki = 1; g.b_n = N;
        g.C = dU; g.c_m = 1; g.c_n = M;
        launch_zgemm_f64(g, nullptr);
        CUDA_OK(cudaDeviceSynchronize());
        CUDA_OK(cudaGetLastError());
        CUDA_OK(cudaMemcpy(U, dU, sizeof(cplx) * (size_t)M * k, cudaMemcpyDeviceToHost));
        CUDA_OK(cudaMemcpy(S, dS, sizeof(double) * k, cudaMemcpyDeviceToHost));
        CUDA_OK(cudaMemcpy(Vh, dVh, sizeof(cplx) * (size_t)k * N, cudaMemcpyDeviceToHost));
        if (discarded) CUDA_OK(cudaMemcpy(discarded, ddisc, sizeof(double), cudaMemcpyDeviceToHost));
        *k_out = k;
    });
}

ttn_status ttn_compress(ttn_ctx* src, ttn_ctx* dst, double* discarded) {
    if (!src || !dst || src == dst || src->Lx != dst->Lx || src->Ly != dst->Ly ||
        src->nodes.size() != dst->nodes.size())
        return TTN_ERR_ARG;
    for (size_t k = 0; k < src->nodes.size(); ++k)
        for (int u = 0; u < 3; ++u)
            if (dst->nodes[k].d[u] > src->nodes[k].d[u]) return TTN_ERR_ARG;
    return guard(dst, [&] {
        ForceFp64 f64;
        ttn_ctx* c = src;
        centre_to_root(c);
        CUDA_OK(cudaStreamSynchronize(c->stream));
        const int nn = (int)c->nodes.size();
        std::vector<void*> temp;
        struct Free {
            std::vector<void*>& t;
            ~Free() {
                for (void* p : t) cudaFree(p);
            }
        } fr{temp};
        auto tmalloc = [&](size_t bytes) {
            void* p = nullptr;
            if (test_take_alloc_fail() || cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess)
                throw TtnError(TTN_ERR_ALLOC, "compress buffers");
            temp.push_back(p);
            return p;
        };
        // bond Grams top-down: G_k(a, a') = <R_a|R_a'>, G_root = [[1]]
        std::vector<cplx*> G(nn, nullptr);
        G[c->root] = (cplx*)tmalloc(sizeof(cplx));
        const cplx one = C(1.0);
        CUDA_OK(cudaMemcpyAsync(G[c->root], &one, sizeof(cplx), cudaMemcpyHostToDevice, c->stream));
        for (int li = (int)c->level_nodes.size() - 1; li >= 0; --li)
            for (int p : c->level_nodes[li]) {
                const Node& np_ = c->nodes[p];
                leg_apply(c, G[p], np_.d[2], c->T[p], np_.d, 2, c->tmp[0], 0.0);
                for (int u = 0; u < 2; ++u) {
                    const int k = np_.child[u];
                    if (k < 0) continue;
                    const long long D = np_.d[u];
                    G[k] = (cplx*)tmalloc(sizeof(cplx) * D * D);
                    project(c, c->T[p], np_.d, c->tmp[0], np_.d, u, G[k], 1, 0, 0);
                }
            }
        // Schmidt bases: one-sided Jacobi on each Gram (Hermitian PSD: its left
        // singular vectors are its eigenvectors), all D columns in descending
        // order; the kept ones are the first D' (their conjugates in the
        // subtree basis)
        unsigned* bar = (unsigned*)tmalloc(sizeof(unsigned) * 4);
        int* err = (int*)tmalloc(sizeof(int) * 4);
        int* info = (int*)tmalloc(sizeof(int) * 4);
        int* order = (int*)tmalloc(sizeof(int) * MAX_CHI);
        int* dk = (int*)tmalloc(sizeof(int) * 4);
        double* ddisc = (double*)tmalloc(sizeof(double));
        double* dS = (double*)tmalloc(sizeof(double) * MAX_CHI);
        cplx* Rw = (cplx*)tmalloc(sizeof(cplx) * MAX_CHI * MAX_CHI);
        cplx* Vw = (cplx*)tmalloc(sizeof(cplx) * MAX_CHI * MAX_CHI);
        cplx* Vh = (cplx*)tmalloc(sizeof(cplx) * MAX_CHI * MAX_CHI);
        std::vector<cplx*> UT(nn, nullptr), UHc(nn, nullptr);   // U^T (no conj) and conj(U)^T per bond
        CUDA_OK(cudaMemsetAsync(err, 0, sizeof(int) * 4, c->stream));
        double dsum = 0.0, dmax = 0.0;
        std::vector<double> hS(MAX_CHI);
        for (int k = 0; k < nn; ++k) {
            if (k == c->root) continue;
            const int D = c->nodes[k].d[2], Dn = dst->nodes[k].d[2];
            CUDA_OK(cudaMemcpyAsync(Rw, G[k], sizeof(cplx) * D * D, cudaMemcpyDeviceToDevice, c->stream));
            if (svd_jacobi_square(Rw, Vw, D, 60, 1e-15, bar, err, info, c->stream) < 0)
                throw TtnError(TTN_ERR_CUDA, "Jacobi launch failed");
            cplx* Ur = (cplx*)tmalloc(sizeof(cplx) * D * D);
            svd_finish(Rw, Vw, D, D, -1.0, Ur, Vh, dS, dk, ddisc, order, c->stream);
            int herr = 0;
            CUDA_OK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            CUDA_OK(cudaMemcpyAsync(hS.data(), dS, sizeof(double) * D, cudaMemcpyDeviceToHost, c->stream));
            CUDA_OK(cudaStreamSynchronize(c->stream));
            if (herr) throw TtnError(TTN_ERR_TIMEOUT, "Jacobi grid barrier wait timed out");
            double tot = 0.0, drop = 0.0;   // eigenvalues of the Gram are its singular values
            for (int t = 0; t < D; ++t) {
                tot += hS[t];
                if (t >= Dn) drop += hS[t];
            }
            const double e = tot > 0.0 ? drop / tot : 0.0;
            dsum += e;
            dmax = std::max(dmax, e);
            // Ur: D x D, its first Dn columns are the kept eigenvectors of G_k;
            // transpose them to Dn x D (the leg matrices below)
            UT[k] = (cplx*)tmalloc(sizeof(cplx) * Dn * D);
            c->stats[3] += k_permute3(Ur, UT[k], D, Dn, 1, 1, 0, 2, 0, c->stream);
        }
        // projected tensors: children legs by U_c^H = Ur_c^T, parent leg by
        // U_k^T = conj(Ur_k)^T, then into dst
        for (int k = 0; k < nn; ++k) {
            const Node& nd = c->nodes[k];
            int d[3] = {nd.d[0], nd.d[1], nd.d[2]};
            const cplx* cur = c->T[k];
            cplx* bufs[2] = {c->tmp[0], c->tmp[1]};
            int bi = 0;
            for (int u = 0; u < 2; ++u) {
                const int ch = nd.child[u];
                if (ch < 0) continue;
                const int Dn = dst->nodes[ch].d[2];
                leg_apply(c, UT[ch], Dn, cur, d, u, bufs[bi], 0.0);
                d[u] = Dn;
                cur = bufs[bi];
                bi ^= 1;
            }
            if (k != c->root) {
                const int Dn = dst->nodes[k].d[2];
                leg_apply(c, UT[k], Dn, cur, d, 2, bufs[bi], 0.0, 1, 0, 0, true);
                d[2] = Dn;
                cur = bufs[bi];
            }
            const long long sz = (long long)d[0] * d[1] * d[2];
            CUDA_OK(cudaMemcpyAsync(dst->T[k], cur, sizeof(cplx) * sz, cudaMemcpyDeviceToDevice, c->stream));
        }
        CUDA_OK(cudaStreamSynchronize(c->stream));
        // canonical form of dst: QR of every non-root node towards its parent, bottom-up
        for (auto& lev : dst->level_nodes)
            for (int k : lev) {
                if (k == dst->root) continue;
                const int p = dst->nodes[k].parent;
                const int u = dst->nodes[p].child[0] == k ? 0 : 1;
                qr_leg(dst, k, 2);
                absorb(dst, p, u, true);
            }
        dst->t = src->t;
        dst->centre = dst->root;
        rebuild_up_envs(dst);
        sync_check(dst);
        if (discarded) {
            discarded[0] = dsum;
            discarded[1] = dmax;
        }
    });
}

// Projective sampling: the depth-first walk of every shot, batched over the
// shots of a batch.  Entering node k with the Gram Gamma_b (parent leg, D x D,
// column-major, trace 1) of shot b's conditioned complement:
//   child 0 : G0_b(c0, c0') = sum_{c1, a, a'} conj X(c0, c1, a) Gamma_b(a, a') X(c0', c1, a')
//             (the c1 subtree is unmeasured and isometric, so it contracts to
//             the identity), walk child 0 -> amplitude vector w0_b(c0);
//   child 1 : Y_b(c1, a) = sum_c0 w0_b(c0) X(c0, c1, a),
//             G1_b(c1, c1') = sum_{a, a'} conj Y_b(c1, a) Gamma_b(a, a') Y_b(c1', a'),
//             walk child 1 -> w1_b(c1);
//   leaving : w_b(a) = sum_c1 w1_b(c1) Y_b(c1, a), normalised.
// A leaf draws from the diagonal of its 3 x 3 Gram and returns e_outcome.
// The root's Gram is [[1]] (its parent leg is the dummy leg of dimension 1).
ttn_status ttn_sample(ttn_ctx* c, const double* uniforms, int n_shots, int* outcomes) {
    if (!c || n_shots < 0 || (n_shots > 0 && (!uniforms || !outcomes))) return TTN_ERR_ARG;
    if (n_shots == 0) return TTN_OK;
    return guard(c, [&] {
        centre_to_root(c);
        const int nn = (int)c->nodes.size(), nl = (int)c->leaf_atom.size(), N = c->N;
        std::vector<int> jidx(nl, -1);   // uniform column of each real leaf
        for (int l = 0, j = 0; l < nl; ++l)
            if (c->leaf_atom[l] >= 0) jidx[l] = j++;
        // per-shot device footprint -> shots per batch (about 2 GB per batch)
        long long per_shot = c->smax + 12LL * nl;
        for (int k = 0; k < nn; ++k) {
            const int* d = c->nodes[k].d;
            per_shot += (long long)d[1] * d[2] + (long long)d[2] * d[2] + d[2];
        }
        const long long budget = 2LL << 30;
        const int S = (int)std::max(1LL, std::min<long long>(n_shots, budget / (16LL * per_shot)));
        std::vector<void*> temp;
        struct Free {
            std::vector<void*>& t;
            ~Free() {
                for (void* p : t) cudaFree(p);
            }
        } fr{temp};
        auto tmalloc = [&](size_t bytes) {
            void* p = nullptr;
            if (test_take_alloc_fail() || cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess)
                throw TtnError(TTN_ERR_ALLOC, "sampling buffers");
            temp.push_back(p);
            return p;
        };
        cplx* Wsc = (cplx*)tmalloc(sizeof(cplx) * (size_t)S * c->smax);
        std::vector<cplx*> gam(nn), Y(nn), wout(nn), lgam(nl), lw(nl);
        for (int k = 0; k < nn; ++k) {
            const int* d = c->nodes[k].d;
            gam[k] = (cplx*)tmalloc(sizeof(cplx) * (size_t)S * d[2] * d[2]);
            Y[k] = (cplx*)tmalloc(sizeof(cplx) * (size_t)S * d[1] * d[2]);
            wout[k] = (cplx*)tmalloc(sizeof(cplx) * (size_t)S * d[2]);
        }
        for (int l = 0; l < nl; ++l) {
            lgam[l] = (cplx*)tmalloc(sizeof(cplx) * 9 * (size_t)S);
            lw[l] = (cplx*)tmalloc(sizeof(cplx) * 3 * (size_t)S);
        }
        double* dU = (double*)tmalloc(sizeof(double) * (size_t)S * N);
        int* dO = (int*)tmalloc(sizeof(int) * (size_t)S * N);
        int nb = 0;   // shots in the current batch
        auto child_gram = [&](const Node& nd, int u) {
            const int ch = nd.child[u];
            return ch >= 0 ? gam[ch] : lgam[-ch - 1];
        };
        std::function<cplx*(int)> visit;
        auto walk_child = [&](const Node& nd, int u) -> cplx* {
            const int ch = nd.child[u];
            if (ch >= 0) return visit(ch);
            const int l = -ch - 1;
            c->stats[3] += k_leaf_draw(lgam[l], dU, N, jidx[l], c->leaf_atom[l], dO, N, lw[l], nb, c->stream);
            return lw[l];
        };
        visit = [&](int k) -> cplx* {
            const Node& nd = c->nodes[k];
            const int d0 = nd.d[0], d1 = nd.d[1], d2 = nd.d[2];
            const long long s = nd.s, d12 = (long long)d1 * d2;
            cplx* G0 = child_gram(nd, 0);
            leg_apply(c, gam[k], d2, c->T[k], nd.d, 2, Wsc, 0.0, nb, (long long)d2 * d2, s);
            project(c, c->T[k], nd.d, Wsc, nd.d, 0, G0, nb, s, (long long)d0 * d0);
            c->stats[3] += k_trace_normalize(G0, d0, (long long)d0 * d0, nb, c->stream);
            const cplx* w0 = walk_child(nd, 0);
            GemmArgs g = base_args();   // Y_b = w0_b x_0 X: (d1 d2) x shots
            g.M = (int)d12; g.N = nb; g.Ki = d0;
            g.A = c->T[k]; g.a_m = d0; g.a_ki = 1;
            g.B = w0; g.b_ki = 1; g.b_n = d0;
            g.C = Y[k]; g.c_m = 1; g.c_n = d12;
            gemm(c, g);
            g = base_args();            // W1_b(c1', a) = sum_a' Y_b(c1', a') Gamma_b(a, a')
            g.M = d1; g.N = d2; g.Ki = d2; g.Bi = nb;
            g.A = Y[k]; g.a_m = 1; g.a_ki = d1; g.a_bi = d12;
            g.B = gam[k]; g.b_ki = d2; g.b_n = 1; g.b_bi = (long long)d2 * d2;
            g.C = Wsc; g.c_m = 1; g.c_n = d1; g.c_bi = d12;
            gemm(c, g);
            cplx* G1 = child_gram(nd, 1);
            g = base_args();            // G1_b(c1, c1') = sum_a conj Y_b(c1, a) W1_b(c1', a)
            g.M = d1; g.N = d1; g.Ki = d2; g.Bi = nb;
            g.A = Y[k]; g.a_m = 1; g.a_ki = d1; g.a_bi = d12; g.conjA = 1;
            g.B = Wsc; g.b_ki = d1; g.b_n = 1; g.b_bi = d12;
            g.C = G1; g.c_m = 1; g.c_n = d1; g.c_bi = (long long)d1 * d1;
            gemm(c, g);
            c->stats[3] += k_trace_normalize(G1, d1, (long long)d1 * d1, nb, c->stream);
            const cplx* w1 = walk_child(nd, 1);
            g = base_args();            // w_b(a) = sum_c1 w1_b(c1) Y_b(c1, a)
            g.M = d2; g.N = 1; g.Ki = d1; g.Bi = nb;
            g.A = Y[k]; g.a_m = d1; g.a_ki = 1; g.a_bi = d12;
            g.B = w1; g.b_ki = 1; g.b_n = d1; g.b_bi = d1;
            g.C = wout[k]; g.c_m = 1; g.c_n = d2; g.c_bi = d2;
            gemm(c, g);
            c->stats[3] += k_vec_normalize(wout[k], d2, d2, nb, c->stream);
            return wout[k];
        };
        for (int b0 = 0; b0 < n_shots; b0 += S) {
            nb = std::min(S, n_shots - b0);
            CUDA_OK(cudaMemcpyAsync(dU, uniforms + (size_t)b0 * N, sizeof(double) * (size_t)nb * N,
                                    cudaMemcpyHostToDevice, c->stream));
            c->stats[3] += k_fill(gam[c->root], nb, C(1.0), c->stream);   // root Gram [[1]] per shot
            visit(c->root);
            CUDA_OK(cudaMemcpyAsync(outcomes + (size_t)b0 * N, dO, sizeof(int) * (size_t)nb * N,
                                    cudaMemcpyDeviceToHost, c->stream));
            CUDA_OK(cudaStreamSynchronize(c->stream));
        }
        sync_check(c);
    });
}

// ---------------------------------------------------------------- gradient
namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the
// Legendre polynomial P_q from the Chebyshev guesses; three-term recurrence).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    for (int i = 0; i < q; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int n = 2; n <= q; ++n) {
                const double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) p0 = 1.0;
            dp = q * (z * p1 - p0) / (z * z - 1.0);   // P_q'(z)
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Device copies of every node tensor of a context (a checkpoint).
struct StateCopy {
    std::vector<cplx*> T;
    double t = 0.0;
};

void save_state(ttn_ctx* c, StateCopy& s, std::vector<void*>& temp) {
    if (s.T.empty()) {
        s.T.resize(c->nodes.size());
        for (size_t k = 0; k < c->nodes.size(); ++k) {
            void* p = nullptr;
            if (test_take_alloc_fail() || cudaMalloc(&p, sizeof(cplx) * c->nodes[k].s) != cudaSuccess)
                throw TtnError(TTN_ERR_ALLOC, "gradient checkpoints");
            temp.push_back(p);
            s.T[k] = (cplx*)p;
        }
    }
    centre_to_root(c);
    for (size_t k = 0; k < c->nodes.size(); ++k)
        CUDA_OK(cudaMemcpyAsync(s.T[k], c->T[k], sizeof(cplx) * c->nodes[k].s, cudaMemcpyDeviceToDevice,
                                c->stream));
    s.t = c->t;
}

// Load a saved state (canonical, centre at the root) and rebuild the upward
// environments.
void load_state(ttn_ctx* c, const StateCopy& s) {
    for (size_t k = 0; k < c->nodes.size(); ++k)
        CUDA_OK(cudaMemcpyAsync(c->T[k], s.T[k], sizeof(cplx) * c->nodes[k].s, cudaMemcpyDeviceToDevice,
                                c->stream));
    c->centre = c->root;
    c->t = s.t;
    rebuild_up_envs(c);
}

// One TDVP step of signed length h with the Hamiltonian at time tm (the
// midpoint of the step being differentiated).
void step_at(ttn_ctx* c, double tm, double h) {
    centre_to_root(c);
    compute_coef(c, tm);
    sweep_fwd(c, c->root, 0.5 * h);
    sweep_rev(c, c->root, 0.5 * h);
    c->t += h;
}

// Transition reduced density matrices of every atom between bra and ket
// (same tree): T_a(s', s) = sum over the other atoms of conj(bra[s', ...])
// ket[s, ...], out[9 a + s' + 3 s] (column-major 3 x 3).  Upward overlap
// environments M_k (bra bond x ket bond) from the leaves, downward ones from
// the root (a leaf's downward environment is its T_a); FP64.
void transition_rdms(ttn_ctx* ket, ttn_ctx* bra, std::vector<zc>& out, std::vector<void*>& temp,
                     std::vector<cplx*>& up, std::vector<cplx*>& dn) {
    ForceFp64 f64;
    ttn_ctx* c = ket;
    const int nn = (int)c->nodes.size();
    auto buf = [&](size_t n) {
        void* p = nullptr;
        if (test_take_alloc_fail() || cudaMalloc(&p, sizeof(cplx) * std::max<size_t>(n, 1)) != cudaSuccess)
            throw TtnError(TTN_ERR_ALLOC, "transition environments");
        temp.push_back(p);
        return (cplx*)p;
    };
    if (up.empty()) {
        up.assign(nn, nullptr);
        dn.assign(nn, nullptr);
        for (int k = 0; k < nn; ++k) {
            const int D = c->nodes[k].d[2];
            up[k] = buf((size_t)D * D);
            dn[k] = buf((size_t)D * D);
        }
        dn.resize(nn + c->n_leaves);
        for (int l = 0; l < c->n_leaves; ++l) dn[nn + l] = buf(9);
    }
    // W = M_{ch0} x_0 ket_k, M_{ch1} x_1 W (leaves: identity), with the
    // legs in `skip` left open
    auto dress = [&](int k, int skip, const cplx*& cur, int* d) {
        const Node& nd = c->nodes[k];
        cur = c->T[k];
        for (int u = 0; u < 3; ++u) d[u] = nd.d[u];
        cplx* bufs[2] = {c->tmp[0], c->tmp[1]};
        int bi = 0;
        for (int u = 0; u < 2; ++u) {
            const int ch = nd.child[u];
            if (ch < 0 || u == skip) continue;
            leg_apply(c, up[ch], nd.d[u], cur, d, u, bufs[bi], 0.0);
            cur = bufs[bi];
            bi ^= 1;
        }
        return bi;
    };
    for (auto& lev : c->level_nodes)
        for (int k : lev) {
            const cplx* cur;
            int d[3];
            dress(k, -1, cur, d);
            project(c, bra->T[k], bra->nodes[k].d, cur, d, 2, up[k], 1, 0, 0);
        }
    // downward: D_root = [[1]]; child u of k: contract bra_k with the other
    // child's M and the parent's D applied to ket_k, leave leg u open
    const cplx one = C(1.0);
    CUDA_OK(cudaMemcpyAsync(dn[c->root], &one, sizeof(cplx), cudaMemcpyHostToDevice, c->stream));
    for (int li = (int)c->level_nodes.size() - 1; li >= 0; --li)
        for (int k : c->level_nodes[li]) {
            const Node& nd = c->nodes[k];
            for (int u = 0; u < 2; ++u) {
                const int ch = nd.child[u];
                const int other = 1 - u;
                const cplx* cur = c->T[k];
                int d[3] = {nd.d[0], nd.d[1], nd.d[2]};
                cplx* bufs[2] = {c->tmp[0], c->tmp[1]};
                int bi = 0;
                if (nd.child[other] >= 0) {
                    leg_apply(c, up[nd.child[other]], nd.d[other], cur, d, other, bufs[bi], 0.0);
                    cur = bufs[bi];
                    bi ^= 1;
                }
                if (k != c->root) {
                    leg_apply(c, dn[k], nd.d[2], cur, d, 2, bufs[bi], 0.0);
                    cur = bufs[bi];
                    bi ^= 1;
                }
                cplx* dst = ch >= 0 ? dn[ch] : dn[nn + (-ch - 1)];
                project(c, bra->T[k], bra->nodes[k].d, cur, d, u, dst, 1, 0, 0);
            }
        }
    std::vector<cplx> h(9 * (size_t)c->n_leaves);
    for (int l = 0; l < c->n_leaves; ++l)
        CUDA_OK(cudaMemcpyAsync(h.data() + 9 * l, dn[nn + l], 9 * sizeof(cplx), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(cudaStreamSynchronize(c->stream));
    out.assign(9 * (size_t)c->N, zc(0.0));
    for (int l = 0; l < c->n_leaves; ++l) {
        const int a = c->leaf_atom[l];
        if (a < 0) continue;
        for (int e = 0; e < 9; ++e) out[9 * (size_t)a + e] = zc(h[9 * l + e].x, h[9 * l + e].y);
    }
}

// A scratch context with c's lattice, bond dimension, Hamiltonian, schedule,
// precision and stream.
ttn_ctx* clone_config(ttn_ctx* c) {
    ttn_ctx* s = nullptr;
    ttn_status st = ttn_create(c->Lx, c->Ly, 3, c->chi, &s);
    if (st != TTN_OK) throw TtnError(st, "gradient: scratch context");
    auto chk = [&](ttn_status r, const char* what) {
        if (r != TTN_OK) {
            std::string m = std::string("gradient: ") + what + ": " + s->err;
            ttn_destroy(s);
            throw TtnError(r, m);
        }
    };
    chk(ttn_set_stream(s, c->stream), "stream");
    chk(ttn_set_precision(s, c->prec), "precision");
    chk(ttn_set_hamiltonian(s, c->xy.data(), c->C6, c->r_cut), "hamiltonian");
    chk(ttn_apply_pulse(s, c->schedule.data(), (int)c->schedule.size()), "pulse");
    return s;
}

}  // namespace

ttn_status ttn_fidelity_gradient(ttn_ctx* c, const ttn_ctx* target, double dt, int n_steps, int n_params,
                                 const int* rows, const int* fields, int n_quad, int checkpoint_every, double* F,
                                 double* grad) {
    if (!c || !target || !F || !(dt > 0.0) || !std::isfinite(dt) || n_steps < 1 || n_params < 0 ||
        (n_params > 0 && (!rows || !fields || !grad)) || n_quad < 1 || n_quad > 8 || target->Lx != c->Lx ||
        target->Ly != c->Ly || target->chi != c->chi || c->gamma != 0.0)
        return TTN_ERR_ARG;
    for (int p = 0; p < n_params; ++p)
        if (rows[p] < 0 || rows[p] >= (int)c->schedule.size() || (fields[p] != 0 && fields[p] != 1))
            return TTN_ERR_ARG;
    ttn_ctx* tgt = const_cast<ttn_ctx*>(target);
    return guard(c, [&] {
        if (tgt->centre != tgt->root) throw TtnError(TTN_ERR_STATE, "target centre is not at its root");
        if (tgt->stream != c->stream) CUDA_OK(cudaStreamSynchronize(tgt->stream));
        std::vector<void*> temp;
        std::vector<ttn_ctx*> scratch;
        struct Free {
            std::vector<void*>& t;
            std::vector<ttn_ctx*>& s;
            ~Free() {
                for (void* p : t) cudaFree(p);
                for (ttn_ctx* x : s) ttn_destroy(x);
            }
        } fr{temp, scratch};
        const int N = n_steps;
        const int L = checkpoint_every > 0 ? checkpoint_every : std::max(1, (int)std::ceil(std::sqrt((double)N)));
        const double t0 = c->t;
        // derivative operators dH/dtheta_p (3 x 3, column-major, |0>,|1>,|r>)
        std::vector<std::array<zc, 9>> E(n_params);
        for (int p = 0; p < n_params; ++p) {
            E[p].fill(zc(0.0));
            const ttn_pulse& row = c->schedule[rows[p]];
            if (fields[p] == 0) {
                const zc e = std::polar(1.0, row.phase_r);
                E[p][2 + 3 * 1] = e;              // |r><1|
                E[p][1 + 3 * 2] = std::conj(e);   // |1><r|
            } else {
                E[p][2 + 3 * 2] = zc(-1.0);       // -|r><r|
            }
        }
        std::vector<double> gx, gw;
        gauss_legendre(n_quad, gx, gw);
        // forward pass with checkpoints every L steps
        StateCopy start;
        save_state(c, start, temp);
        std::vector<StateCopy> cps((N + L - 1) / L);
        for (int n = 0; n < N; ++n) {
            if (n % L == 0) save_state(c, cps[n / L], temp);
            step_at(c, t0 + (n + 0.5) * dt, dt);
        }
        const zc A = overlap(c, tgt);
        std::vector<double> g(n_params, 0.0);
        if (n_params > 0) {
            ttn_ctx* chi = clone_config(c);
            scratch.push_back(chi);
            ttn_ctx* pw = clone_config(c);
            scratch.push_back(pw);
            ttn_ctx* cw = clone_config(c);
            scratch.push_back(cw);
            // chi_N = target
            for (size_t k = 0; k < c->nodes.size(); ++k)
                CUDA_OK(cudaMemcpyAsync(chi->T[k], tgt->T[k], sizeof(cplx) * c->nodes[k].s, cudaMemcpyDeviceToDevice,
                                        c->stream));
            chi->centre = chi->root;
            chi->t = t0 + N * dt;
            rebuild_up_envs(chi);
            std::vector<StateCopy> seg(L);
            StateCopy chis;
            std::vector<zc> T;
            std::vector<cplx*> up, dn;
            for (int cp = (int)cps.size() - 1; cp >= 0; --cp) {
                // states psi_{cp L} .. psi_{cp L + len - 1} of this segment
                const int n0 = cp * L, len = std::min(L, N - n0);
                load_state(c, cps[cp]);
                for (int i = 0; i < len; ++i) {
                    save_state(c, seg[i], temp);
                    if (i + 1 < len) step_at(c, t0 + (n0 + i + 0.5) * dt, dt);
                }
                for (int i = len - 1; i >= 0; --i) {
                    const int n = n0 + i;               // step n: psi_n -> psi_{n+1}
                    const double tm = t0 + (n + 0.5) * dt;
                    std::vector<int> act;
                    for (int p = 0; p < n_params; ++p) {
                        const ttn_pulse& row = c->schedule[rows[p]];
                        if (row.t0 <= tm && tm < row.t1) act.push_back(p);
                    }
                    if (!act.empty()) {
                        save_state(chi, chis, temp);
                        std::vector<zc> acc(n_params, zc(0.0));
                        for (int j = 0; j < n_quad; ++j) {
                            const double sj = 0.5 * dt * (1.0 + gx[j]);
                            load_state(pw, seg[i]);
                            step_at(pw, tm, sj);                 // psi(s_j)
                            load_state(cw, chis);
                            step_at(cw, tm, -(dt - sj));         // chi(s_j)
                            transition_rdms(pw, cw, T, temp, up, dn);
                            for (int p : act) {
                                const int a = c->schedule[rows[p]].atom;
                                zc v(0.0);
                                for (int e = 0; e < 9; ++e) v += E[p][e] * T[9 * (size_t)a + e];
                                acc[p] += 0.5 * dt * gw[j] * v;
                            }
                        }
                        for (int p : act) g[p] += 2.0 * (std::conj(A) * (zc(0.0, -1.0) * acc[p])).real();
                    }
                    step_at(chi, tm, -dt);                      // chi_n = U_{n+1}^H chi_{n+1}
                }
            }
        }
        // restore the context's state and time
        load_state(c, start);
        sync_check(c);
        *F = std::norm(A);
        for (int p = 0; p < n_params; ++p) grad[p] = g[p];
    });
}

ttn_status ttn_test_inject(int kind, long long value) {
    if (value < 0) return TTN_ERR_ARG;
    switch (kind) {
        case TTN_INJECT_NONE:
            g_inj_tc_stall = 0;
            g_inj_mmax = 0;
            g_inj_alloc_fail = 0;
            return TTN_OK;
        case TTN_INJECT_TC_STALL: g_inj_tc_stall = value; return TTN_OK;
        case TTN_INJECT_KRYLOV_MMAX:
            if (value > KRYLOV_MMAX) return TTN_ERR_ARG;
            g_inj_mmax = (int)value;
            return TTN_OK;
        case TTN_INJECT_ALLOC_FAIL: g_inj_alloc_fail = value; return TTN_OK;
        default: return TTN_ERR_ARG;
    }
}

ttn_status ttn_profile_records(const ttn_ctx* c, double* out, int max_records, int* n_records) {
    if (!c || !n_records) return TTN_ERR_ARG;
    *n_records = (int)c->prof_last.size();
    if (out)
        for (int i = 0; i < std::min(max_records, *n_records); ++i)
            for (int j = 0; j < 7; ++j) out[7 * i + j] = c->prof_last[i][j];
    return TTN_OK;
}

ttn_status ttn_get_stats(const ttn_ctx* c, int64_t* out) {
    if (!c || !out) return TTN_ERR_ARG;
    for (int i = 0; i < 6; ++i) out[i] = c->stats[i];
    std::memcpy(&out[2], &c->max_err, sizeof(double));
    return TTN_OK;
}

ttn_status ttn_reset_stats(ttn_ctx* c) {
    if (!c) return TTN_ERR_ARG;
    for (int i = 0; i < 6; ++i) c->stats[i] = 0;
    c->max_err = 0.0;
    return TTN_OK;
}

}  // extern "C"
