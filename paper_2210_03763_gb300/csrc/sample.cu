// Kernels of the projective measurement sampler (ttn_sample): the per-shot
// normalisations of the depth-first walk and the draw at a leaf.  The walk's
// contractions are ordinary batched GEMMs (one batch entry per shot).
//
// Measurement in the {|0>, |1>, |r>} basis of every atom, atoms in leaf
// order, each outcome drawn from its conditional distribution given the
// outcomes already drawn (Sec. "Parallel quantum algorithms", measurement
// histograms): the draw is inverse transform sampling with a uniform number
// supplied by the caller, outcome s = the first level with
// u < (P(0) + ... + P(s)) / (P(0) + P(1) + P(2)).
#include "common.cuh"

namespace {

constexpr int NT = 256;

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) t += sh[i];
    __syncthreads();
    return t;
}

// G_b <- G_b / max(Re tr G_b, 1e-300) for the D x D matrices of S shots
// (stride ld complex); one block per shot.
__global__ void __launch_bounds__(NT) trace_normalize_kernel(cplx* G, int D, long long ld) {
    __shared__ double sh[NT / 32];
    __shared__ double sfac;
    cplx* g = G + blockIdx.x * ld;
    double t = 0.0;
    for (int i = threadIdx.x; i < D; i += NT) t += g[(long long)i * (D + 1)].x;
    t = block_sum(t, sh);
    if (threadIdx.x == 0) sfac = 1.0 / fmax(t, 1e-300);
    __syncthreads();
    const double f = sfac;
    for (long long e = threadIdx.x; e < (long long)D * D; e += NT) {
        cplx v = g[e];
        g[e] = make_double2(v.x * f, v.y * f);
    }
}

// w_b <- w_b / |w_b| (unchanged when zero) for S vectors of length D.
__global__ void __launch_bounds__(NT) vec_normalize_kernel(cplx* w, int D, long long ld) {
    __shared__ double sh[NT / 32];
    __shared__ double sfac;
    cplx* x = w + blockIdx.x * ld;
    double t = 0.0;
    for (int i = threadIdx.x; i < D; i += NT) t += x[i].x * x[i].x + x[i].y * x[i].y;
    t = block_sum(t, sh);
    if (threadIdx.x == 0) sfac = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
    __syncthreads();
    const double f = sfac;
    for (int i = threadIdx.x; i < D; i += NT) x[i] = make_double2(x[i].x * f, x[i].y * f);
}

// Leaf of atom `atom` (-1: padding, always |0>, no uniform consumed): shot b
// draws s from the diagonal of its 3 x 3 Gram G_b with u = U[b * ldu + j];
// outcome into out[b * N + atom]; w_b = e_s.
__global__ void leaf_draw_kernel(const cplx* G, const double* U, long long ldu, int j, int atom, int* out, int N,
                                 cplx* w, int S) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= S) return;
    int s = 0;
    if (atom >= 0) {
        const cplx* g = G + 9LL * b;
        const double p0 = fmax(g[0].x, 0.0), p1 = fmax(g[4].x, 0.0), p2 = fmax(g[8].x, 0.0);
        const double c1 = p0 + p1, tot = c1 + p2;
        const double u = U[b * ldu + j];
        if (tot > 0.0) {
            if (u < p0 / tot) s = 0;
            else if (u < c1 / tot) s = 1;
            else s = 2;
        } else {
            s = 0;    // an all-zero distribution (zero state): the first level
        }
        out[(long long)b * N + atom] = s;
    }
    cplx* x = w + 3LL * b;
    for (int i = 0; i < 3; ++i) x[i] = make_double2(i == s ? 1.0 : 0.0, 0.0);
}

}  // namespace

int k_trace_normalize(cplx* G, int D, long long ld, int S, cudaStream_t s) {
    if (S <= 0) return 0;
    trace_normalize_kernel<<<S, NT, 0, s>>>(G, D, ld);
    return 1;
}

int k_vec_normalize(cplx* w, int D, long long ld, int S, cudaStream_t s) {
    if (S <= 0) return 0;
    vec_normalize_kernel<<<S, NT, 0, s>>>(w, D, ld);
    return 1;
}

int k_leaf_draw(const cplx* G, const double* U, long long ldu, int j, int atom, int* out, int N, cplx* w, int S,
                cudaStream_t s) {
    if (S <= 0) return 0;
    leaf_draw_kernel<<<(S + 127) / 128, 128, 0, s>>>(G, U, ldu, j, atom, out, N, w, S);
    return 1;
}
