// Thomas modified-coefficient precompute (FP64, on the GPU), once per
// create.  The line matrices are constant along every line of an axis, so
// the elimination pivots depend only on (substrate, axis, position).
//
// Plain form (used by the FP32 field and the plain FP64 sweep):
//   forward   d'_0 = d_0 r_0,  d'_i = (d_i + c d'_{i-1}) r_i,   r_i = 1/den_i
//   backward  x_{n-1} = d'_{n-1},  x_i = d'_i + (c r_i) x_{i+1}
//
// Rescaled form (FP64): with w_i = den_i d'_i and z_i = den_i x_i the two
// recurrences become one FMA each,
//   w_i = d_i + (c r_{i-1}) w_{i-1},   z_i = w_i + (c r_{i+1}) z_{i+1},
// and the output is the solution times den_i.  If the input already carries
// a per-position scale sigma_i along the axis (from earlier sweeps) the same
// two FMAs absorb it with coefficients
//   fa_i = c r_{i-1} sigma_i / sigma_{i-1},  fb_i = c r_{i+1} sigma_i / sigma_{i+1},
// and the output scale is sigma_i den_i.  State p of an axis has
// sigma = den^p; after `period` steps the z sweep divides the whole scale
// out again.  A factor constant along a line (the other axes' scales) passes
// through a linear solve untouched, which is what keeps the scale separable.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace bfvm {

namespace {

struct CoefParams {
    int n[3];
    int off[3];
    int L;
    int n_sub;
    int dims;          // 3, or 2 for the 2-D variant (decay share lambda dt / dims per axis)
    double dx, dt;
    const double* D;
    const double* lambda;
};

// One thread per (substrate, axis): the sequential pivot recurrence.
__global__ void k_pivots(CoefParams P, double* r, double* cr, double* cvec,
                         double* den_out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.n_sub * 3) return;
    int s = t / 3, a = t % 3;
    int n = P.n[a];
    double c = P.D[s] * P.dt / (P.dx * P.dx);
    double ell = P.lambda[s] * P.dt / (double)P.dims;
    cvec[s * 3 + a] = c;
    int64_t base = (int64_t)s * P.L + P.off[a];
    double den_prev = 1.0;
    for (int i = 0; i < n; ++i) {
        int nb = (i > 0) + (i < n - 1);
        double b = 1.0 + ell + c * (double)nb;
        double den = (i == 0) ? b : b - c * (c / den_prev);
        den_out[base + i] = den;
        r[base + i] = 1.0 / den;
        cr[base + i] = c / den;
        den_prev = den;
    }
}

// hi/lo float split: b[i] = fl32(a[i]), b[n + i] = fl32(a[i] - b[i])
__global__ void k_split32(const double* a, float* b, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hi = (float)a[i];
    b[i] = hi;
    b[n + i] = (float)(a[i] - (double)hi);
}

// One thread per (substrate, axis, position): scale vectors of all states.
__global__ void k_scales(int64_t n_entries, int period, const double* den,
                         double* sc, double* isc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_entries) return;
    double s = 1.0;
    double d = den[e];
    for (int p = 0; p <= period; ++p) {
        sc[(int64_t)p * n_entries + e] = s;
        isc[(int64_t)p * n_entries + e] = 1.0 / s;
        s *= d;
    }
}

// One thread per (state, substrate, axis, position): fa, fb of that state.
__global__ void k_scaled_coefs(CoefParams P, int period, const double* r,
                               const double* sc, const double* isc,
                               double* fa, double* fb)
{
    int64_t per_state = (int64_t)P.n_sub * P.L;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= per_state * period) return;
    int p = (int)(e / per_state);
    int64_t q = e % per_state;
    int s = (int)(q / P.L);
    int pos = (int)(q % P.L);
    int a = pos < P.off[1] ? 0 : (pos < P.off[2] ? 1 : 2);
    int i = pos - P.off[a];
    int n = P.n[a];
    double c = P.D[s] * P.dt / (P.dx * P.dx);
    const double* scp = sc + (int64_t)p * per_state;
    const double* iscp = isc + (int64_t)p * per_state;
    fa[e] = (i > 0) ? c * r[q - 1] * (scp[q] * iscp[q - 1]) : 0.0;
    fb[e] = (i < n - 1) ? c * r[q + 1] * (scp[q] * iscp[q + 1]) : 0.0;
}

}  // namespace

// Number of steps between rescales: the stored field may grow by at most
// prod_axes max_i den_i per step; keep that product below 1e200 so that
// fields up to 1e100 in magnitude stay far from overflow.  den_i <= b_i <=
// 1 + ell + 2c bounds it from the inputs alone.
static int rescale_period(const Ctx* c)
{
    double worst = 0.0;
    for (int s = 0; s < c->n_sub; ++s) {
        double cc = c->D[s] * c->dt / (c->dx * c->dx);
        double ell = c->lambda[s] * c->dt / (double)c->dims;
        double g = 3.0 * log10(1.0 + ell + 2.0 * cc);
        if (g > worst) worst = g;
    }
    int m = worst > 0.0 ? (int)floor(200.0 / worst) : 64;
    if (m > 64) m = 64;
    if (m < 1) m = 1;
    if (c->period_override > 0) m = c->period_override;
    return m;
}

// Split line solve: prefix and suffix products of cr within the segments of
// one axis, one thread per (substrate, segment), in FP64.
__global__ void k_split_products(const double* cr, double* sg, double* sl, int n_sub,
                                 int64_t L, int off, int n, int m)
{
    const int n_seg = (n + m - 1) / m;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_sub * n_seg) return;
    const int s = t / n_seg, q = t % n_seg;
    const int k0 = q * m, k1 = min(n, k0 + m);
    const int64_t row = (int64_t)s * L + off;
    double p = 1.0;
    for (int k = k0; k < k1; ++k) {
        p *= cr[row + k];
        sg[row + k] = p;
    }
    p = 1.0;
    for (int k = k1 - 1; k >= k0; --k) {
        p *= cr[row + k];
        sl[row + k] = p;
    }
}

// Segment length of the split solve along an axis with n elements per line
// and `lines` lines: enough segments for about 1024 threads per SM, at most
// 64 segments unless that makes them longer than 64 elements (the x tile),
// at least 8 elements each.
int split_segment_length(int n, int64_t lines, int sm_count)
{
    const int64_t target = (int64_t)std::max(sm_count, 1) * 1024;
    int64_t P = (target + lines - 1) / std::max<int64_t>(lines, 1);
    if (P > 64) P = 64;
    if (P < 1) P = 1;
    int m = (int)((n + P - 1) / P);
    if (m > 64) m = 64;
    if (m < 8) m = 8;
    if (m > n) m = n;
    return std::max(m, 1);
}

bfvm_status build_coefficients(Ctx* c)
{
    free_coefficients(c);
    CoefTables& T = c->coef;
    T.L = (int64_t)c->nx + c->ny + c->nz;
    int64_t n_tab = (int64_t)c->n_sub * T.L;
    CoefParams P;
    P.n[0] = c->nx; P.n[1] = c->ny; P.n[2] = c->nz;
    P.off[0] = 0; P.off[1] = c->nx; P.off[2] = c->nx + c->ny;
    P.L = (int)T.L;
    P.n_sub = c->n_sub;
    P.dx = c->dx;
    P.dt = c->dt;
    double *dD = nullptr, *dl = nullptr, *den = nullptr;
    BFVM_CUDA(c, cudaMalloc(&dD, sizeof(double) * c->n_sub));
    BFVM_CUDA(c, cudaMalloc(&dl, sizeof(double) * c->n_sub));
    BFVM_CUDA(c, cudaMemcpyAsync(dD, c->D.data(), sizeof(double) * c->n_sub,
                                 cudaMemcpyHostToDevice, c->stream));
    BFVM_CUDA(c, cudaMemcpyAsync(dl, c->lambda.data(), sizeof(double) * c->n_sub,
                                 cudaMemcpyHostToDevice, c->stream));
    P.D = dD;
    P.lambda = dl;
    P.dims = c->dims;
    BFVM_CUDA(c, cudaMalloc(&T.r, sizeof(double) * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.cr, sizeof(double) * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.c, sizeof(double) * c->n_sub * 3));
    BFVM_CUDA(c, cudaMalloc(&den, sizeof(double) * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.r32, sizeof(float) * 2 * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.cr32, sizeof(float) * 2 * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.c32, sizeof(float) * 2 * c->n_sub * 3));
    int nt = c->n_sub * 3;
    k_pivots<<<(nt + 63) / 64, 64, 0, c->stream>>>(P, T.r, T.cr, T.c, den);
    BFVM_CUDA(c, cudaGetLastError());
    int blk = 256;
    k_split32<<<ceil_div(n_tab, blk), blk, 0, c->stream>>>(T.r, T.r32, n_tab);
    k_split32<<<ceil_div(n_tab, blk), blk, 0, c->stream>>>(T.cr, T.cr32, n_tab);
    k_split32<<<1, 64, 0, c->stream>>>(T.c, T.c32, c->n_sub * 3);
    BFVM_CUDA(c, cudaGetLastError());
    c->launches += 4;

    // split line solve tables and exchange buffer
    BFVM_CUDA(c, cudaMalloc(&T.sg, sizeof(double) * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.sl, sizeof(double) * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.sg32, sizeof(float) * 2 * n_tab));
    BFVM_CUDA(c, cudaMalloc(&T.sl32, sizeof(float) * 2 * n_tab));
    {
        const int ext[3] = {c->nx, c->ny, c->nz};
        int64_t ex_elems = 0;
        for (int a = 0; a < 3; ++a) {
            const int64_t lines = (int64_t)ext[0] * ext[1] * ext[2] / ext[a] * c->n_sub;
            const int m = split_segment_length(ext[a], lines, c->sm_count);
            T.seg[a] = m;
            const int n_seg = (ext[a] + m - 1) / m;
            ex_elems = std::max(ex_elems, 2 * lines * n_seg);
            const int nt_s = c->n_sub * n_seg;
            k_split_products<<<ceil_div(nt_s, 64), 64, 0, c->stream>>>(T.cr, T.sg, T.sl, c->n_sub,
                                                                       T.L, P.off[a], ext[a], m);
            c->launches += 1;
        }
        BFVM_CUDA(c, cudaGetLastError());
        k_split32<<<ceil_div(n_tab, blk), blk, 0, c->stream>>>(T.sg, T.sg32, n_tab);
        k_split32<<<ceil_div(n_tab, blk), blk, 0, c->stream>>>(T.sl, T.sl32, n_tab);
        BFVM_CUDA(c, cudaGetLastError());
        c->launches += 2;
        const size_t esz = c->precision == 64 ? sizeof(double) : sizeof(float);
        BFVM_CUDA(c, cudaMalloc(&T.split_ex, esz * (size_t)std::max<int64_t>(ex_elems, 1)));
    }

    if (c->precision == 64) {
        int m = rescale_period(c);
        T.period = m;
        BFVM_CUDA(c, cudaMalloc(&T.sc, sizeof(double) * n_tab * (m + 1)));
        BFVM_CUDA(c, cudaMalloc(&T.isc, sizeof(double) * n_tab * (m + 1)));
        BFVM_CUDA(c, cudaMalloc(&T.fa, sizeof(double) * n_tab * m));
        BFVM_CUDA(c, cudaMalloc(&T.fb, sizeof(double) * n_tab * m));
        k_scales<<<ceil_div(n_tab, blk), blk, 0, c->stream>>>(n_tab, m, den, T.sc, T.isc);
        k_scaled_coefs<<<ceil_div(n_tab * m, blk), blk, 0, c->stream>>>(
            P, m, T.r, T.sc, T.isc, T.fa, T.fb);
        BFVM_CUDA(c, cudaGetLastError());
        c->launches += 2;
    }
    BFVM_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(dD);
    cudaFree(dl);
    cudaFree(den);
    return BFVM_OK;
}

void free_coefficients(Ctx* c)
{
    CoefTables& T = c->coef;
    void* ptrs[] = {T.r, T.cr, T.c, T.r32, T.cr32, T.c32, T.fa, T.fb, T.sc, T.isc,
                    T.sg, T.sl, T.sg32, T.sl32, T.split_ex};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    T = CoefTables();
}

}  // namespace bfvm
