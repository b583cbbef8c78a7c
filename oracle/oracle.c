/*
 * Plain FP64 CPU oracle for the substrate diffusion-decay-source step of
 * Eq. (1) ("Introduction and Motivation"), solved as BioFVM's locally
 * one-dimensional (LOD) implicit finite-volume update ("Using OpenACC
 * programming model for PhysiCell": x-, y- and z-diffusion per step;
 * "Elements of Parallelism": Dirichlet conditions applied on the device).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * It is deliberately slow and literal:
 *   - every line solve gathers the line into a buffer, builds the line
 *     matrix and runs the textbook Thomas algorithm with divisions;
 *   - the step is: Dirichlet, x-solve, Dirichlet, y-solve, Dirichlet,
 *     z-solve, Dirichlet, then every cell in ascending index order updates
 *     its own voxel with the implicit source formula.
 * Independent lines of one sweep may run on several OpenMP threads; that
 * changes no arithmetic.
 *
 * Field layout: rho[s][z][y][x], x fastest, one contiguous block per
 * substrate.  All numbers are FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Line matrix of one axis (Eq. 1, diffusion + decay, implicit Euler,  */
/* LOD share lambda*dt/3 of the decay per axis).                       */
/*                                                                      */
/* Cell-centred finite volumes with zero-flux faces: with              */
/* c = D dt / dx^2 and ell = lambda dt / 3,                            */
/*   n == 1 : A = [1 + ell]                                             */
/*   n >= 2 : diag 1+ell+c at both ends, 1+ell+2c inside,               */
/*            off-diagonals -c.                                         */
/* ------------------------------------------------------------------ */
void oracle_line_matrix(int n, double c, double ell,
                        double* lower, double* diag, double* upper)
{
    for (int i = 0; i < n; ++i) {
        int left = (i > 0);
        int right = (i < n - 1);
        diag[i] = 1.0 + ell + c * (double)(left + right);
        lower[i] = left ? -c : 0.0;
        upper[i] = right ? -c : 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Textbook Thomas algorithm for a general tridiagonal system          */
/*   lower[i] x[i-1] + diag[i] x[i] + upper[i] x[i+1] = rhs[i].        */
/* Forward elimination then back substitution, with plain divisions.   */
/* `work` holds n doubles.                                              */
/* ------------------------------------------------------------------ */
void oracle_tridiag_solve(int n, const double* lower, const double* diag,
                          const double* upper, const double* rhs,
                          double* x, double* work)
{
    double* cprime = work;          /* modified upper coefficients */
    double denom = diag[0];
    cprime[0] = upper[0] / denom;
    x[0] = rhs[0] / denom;
    for (int i = 1; i < n; ++i) {
        denom = diag[i] - lower[i] * cprime[i - 1];
        cprime[i] = upper[i] / denom;
        x[i] = (rhs[i] - lower[i] * x[i - 1]) / denom;
    }
    for (int i = n - 2; i >= 0; --i)
        x[i] = x[i] - cprime[i] * x[i + 1];
}

static int64_t vox_index(int nx, int ny, int nz, int s, int z, int y, int x)
{
    return (((int64_t)s * nz + z) * ny + y) * (int64_t)nx + x;
}

/* ------------------------------------------------------------------ */
/* Dirichlet condition ("apply-dirichlet-conditions", Elements of      */
/* Parallelism): every voxel of the outermost layer on all six faces   */
/* of a Dirichlet substrate is set to that substrate's value.          */
/* ------------------------------------------------------------------ */
void oracle_apply_dirichlet(int nx, int ny, int nz, int n_sub,
                            const int* bc_kind, const double* bc_value,
                            double* rho)
{
    for (int s = 0; s < n_sub; ++s) {
        if (bc_kind[s] != 1) continue;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int on_shell = (x == 0 || x == nx - 1 || y == 0 ||
                                    y == ny - 1 || z == 0 || z == nz - 1);
                    if (on_shell)
                        rho[vox_index(nx, ny, nz, s, z, y, x)] = bc_value[s];
                }
    }
}

/* Jacobian of the Dirichlet projection: zero on the shell of Dirichlet
 * substrates (the value there no longer depends on the input). */
static void project_dirichlet_adjoint(int nx, int ny, int nz, int n_sub,
                                      const int* bc_kind, double* g)
{
    double zero[1] = {0.0};
    (void)zero;
    for (int s = 0; s < n_sub; ++s) {
        if (bc_kind[s] != 1) continue;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int on_shell = (x == 0 || x == nx - 1 || y == 0 ||
                                    y == ny - 1 || z == 0 || z == nz - 1);
                    if (on_shell) g[vox_index(nx, ny, nz, s, z, y, x)] = 0.0;
                }
    }
}

/* ------------------------------------------------------------------ */
/* One implicit solve along `axis` (0 = x, 1 = y, 2 = z) for every     */
/* line of every substrate: rho <- A_axis^{-1} rho.  Each line is      */
/* gathered, solved with oracle_tridiag_solve and scattered back.      */
/* ------------------------------------------------------------------ */
void oracle_axis_solve(int axis, int nx, int ny, int nz, int n_sub,
                       double dx, double dt, const double* D,
                       const double* lambda, double* rho, int n_threads)
{
    int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
    int64_t stride = axis == 0 ? 1 : (axis == 1 ? (int64_t)nx : (int64_t)nx * ny);
    int n_a = axis == 0 ? ny : nx;      /* first "other" extent */
    int n_b = axis == 2 ? ny : nz;      /* second "other" extent */
    int64_t n_lines_per_sub = (int64_t)n_a * n_b;

    for (int s = 0; s < n_sub; ++s) {
        double c = D[s] * dt / (dx * dx);
        double ell = lambda[s] * dt / 3.0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads > 0 ? n_threads : 1)
#endif
        {
            double* buf = (double*)malloc(sizeof(double) * 6 * (size_t)n_axis);
            double* lower = buf;
            double* diag = buf + n_axis;
            double* upper = buf + 2 * n_axis;
            double* rhs = buf + 3 * n_axis;
            double* x = buf + 4 * n_axis;
            double* work = buf + 5 * n_axis;
            oracle_line_matrix(n_axis, c, ell, lower, diag, upper);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int64_t line = 0; line < n_lines_per_sub; ++line) {
                int a = (int)(line % n_a);
                int b = (int)(line / n_a);
                int64_t base;
                if (axis == 0)      base = vox_index(nx, ny, nz, s, b, a, 0);
                else if (axis == 1) base = vox_index(nx, ny, nz, s, b, 0, a);
                else                base = vox_index(nx, ny, nz, s, 0, b, a);
                for (int i = 0; i < n_axis; ++i) rhs[i] = rho[base + i * stride];
                oracle_tridiag_solve(n_axis, lower, diag, upper, rhs, x, work);
                for (int i = 0; i < n_axis; ++i) rho[base + i * stride] = x[i];
            }
            free(buf);
        }
        (void)n_threads;
    }
}

/* Voxel of a cell (cell-centred grid, origin 0): v_a = floor(p_a / dx),
 * clamped to n_a - 1 so that a cell on the upper domain face belongs to the
 * last voxel. */
int64_t oracle_cell_voxel(int nx, int ny, int nz, double dx, const double* p)
{
    int n[3] = {nx, ny, nz};
    int v[3];
    for (int a = 0; a < 3; ++a) {
        double q = floor(p[a] / dx);
        int64_t qi = (int64_t)q;
        if (qi > n[a] - 1) qi = n[a] - 1;
        if (qi < 0) qi = 0;
        v[a] = (int)qi;
    }
    return ((int64_t)v[2] * ny + v[1]) * (int64_t)nx + v[0];
}

/* ------------------------------------------------------------------ */
/* Cell sources and sinks (the delta-function term of Eq. 1), implicit */
/* in time: for each cell i in ascending index order, in its voxel v,  */
/* for each substrate,                                                  */
/*   rho_v <- (rho_v + dt (V_i/V_vox) S_i rho*_i)                       */
/*            / (1 + dt (V_i/V_vox) (S_i + U_i)),   V_vox = dx^3.       */
/* ------------------------------------------------------------------ */
void oracle_apply_sources(int nx, int ny, int nz, int n_sub, double dx,
                          double dt, int64_t n_cells, const double* pos,
                          const double* vol, const double* S, const double* U,
                          const double* rho_star, double* rho)
{
    double v_vox = dx * dx * dx;
    int64_t n_vox = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < n_cells; ++i) {
        int64_t v = oracle_cell_voxel(nx, ny, nz, dx, pos + 3 * i);
        double w = dt * (vol[i] / v_vox);
        for (int s = 0; s < n_sub; ++s) {
            double a = w * S[i * n_sub + s] * rho_star[i * n_sub + s];
            double b = w * (S[i * n_sub + s] + U[i * n_sub + s]);
            double* r = rho + (int64_t)s * n_vox + v;
            *r = (*r + a) / (1.0 + b);
        }
    }
}

/* One full LOD step, in the order Dirichlet, x, Dirichlet, y, Dirichlet,
 * z, Dirichlet, sources. */
void oracle_step(int nx, int ny, int nz, double dx, double dt, int n_sub,
                 const double* D, const double* lambda, const int* bc_kind,
                 const double* bc_value, int64_t n_cells, const double* pos,
                 const double* vol, const double* S, const double* U,
                 const double* rho_star, double* rho, int n_threads)
{
    oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, rho);
    for (int axis = 0; axis < 3; ++axis) {
        oracle_axis_solve(axis, nx, ny, nz, n_sub, dx, dt, D, lambda, rho, n_threads);
        oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, rho);
    }
    oracle_apply_sources(nx, ny, nz, n_sub, dx, dt, n_cells, pos, vol, S, U,
                         rho_star, rho);
}

/* n_steps full steps, in place on rho. */
int oracle_run(int nx, int ny, int nz, double dx, double dt, int n_sub,
               const double* D, const double* lambda, const int* bc_kind,
               const double* bc_value, int64_t n_cells, const double* pos,
               const double* vol, const double* S, const double* U,
               const double* rho_star, int n_steps, int n_threads, double* rho)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_sub < 1 || n_steps < 0) return 1;
    for (int t = 0; t < n_steps; ++t)
        oracle_step(nx, ny, nz, dx, dt, n_sub, D, lambda, bc_kind, bc_value,
                    n_cells, pos, vol, S, U, rho_star, rho, n_threads);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 2-D variant (the paper also ports BioFVM's 2-D diffusion: x- and    */
/* y-diffusion only, "Using OpenACC programming model for PhysiCell"). */
/* The grid is nx x ny x 1.  Each of the two axes takes half of the    */
/* decay, ell = lambda dt / 2; the Dirichlet shell is the outer layer  */
/* of the four edges x = 0, nx-1 and y = 0, ny-1 (the single z layer   */
/* is not a boundary).  Step: Dirichlet, x-solve, Dirichlet, y-solve,  */
/* Dirichlet, sources (V_vox = dx^3 as in 3-D).                        */
/* ------------------------------------------------------------------ */
void oracle_apply_dirichlet_2d(int nx, int ny, int n_sub, const int* bc_kind,
                               const double* bc_value, double* rho)
{
    for (int s = 0; s < n_sub; ++s) {
        if (bc_kind[s] != 1) continue;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)
                    rho[vox_index(nx, ny, 1, s, 0, y, x)] = bc_value[s];
    }
}

/* One implicit solve along axis 0 (x) or 1 (y) of a 2-D grid with the
 * 2-D decay share lambda dt / 2. */
void oracle_axis_solve_2d(int axis, int nx, int ny, int n_sub, double dx, double dt,
                          const double* D, const double* lambda, double* rho)
{
    const int n_axis = axis == 0 ? nx : ny;
    const int n_other = axis == 0 ? ny : nx;
    const int64_t stride = axis == 0 ? 1 : (int64_t)nx;
    double* buf = (double*)malloc(sizeof(double) * 6 * (size_t)n_axis);
    double* lower = buf;
    double* diag = buf + n_axis;
    double* upper = buf + 2 * n_axis;
    double* rhs = buf + 3 * n_axis;
    double* x = buf + 4 * n_axis;
    double* work = buf + 5 * n_axis;
    for (int s = 0; s < n_sub; ++s) {
        double c = D[s] * dt / (dx * dx);
        double ell = lambda[s] * dt / 2.0;
        oracle_line_matrix(n_axis, c, ell, lower, diag, upper);
        for (int o = 0; o < n_other; ++o) {
            int64_t base = axis == 0 ? vox_index(nx, ny, 1, s, 0, o, 0)
                                     : vox_index(nx, ny, 1, s, 0, 0, o);
            for (int i = 0; i < n_axis; ++i) rhs[i] = rho[base + i * stride];
            oracle_tridiag_solve(n_axis, lower, diag, upper, rhs, x, work);
            for (int i = 0; i < n_axis; ++i) rho[base + i * stride] = x[i];
        }
    }
    free(buf);
}

/* n_steps 2-D steps in place on rho (nz must be 1). */
int oracle_run_2d(int nx, int ny, int nz, double dx, double dt, int n_sub,
                  const double* D, const double* lambda, const int* bc_kind,
                  const double* bc_value, int64_t n_cells, const double* pos,
                  const double* vol, const double* S, const double* U,
                  const double* rho_star, int n_steps, int n_threads, double* rho)
{
    (void)n_threads;
    if (nx < 1 || ny < 1 || nz != 1 || n_sub < 1 || n_steps < 0) return 1;
    for (int t = 0; t < n_steps; ++t) {
        oracle_apply_dirichlet_2d(nx, ny, n_sub, bc_kind, bc_value, rho);
        for (int axis = 0; axis < 2; ++axis) {
            oracle_axis_solve_2d(axis, nx, ny, n_sub, dx, dt, D, lambda, rho);
            oracle_apply_dirichlet_2d(nx, ny, n_sub, bc_kind, bc_value, rho);
        }
        oracle_apply_sources(nx, ny, 1, n_sub, dx, dt, n_cells, pos, vol, S, U,
                             rho_star, rho);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Dirichlet nodes inside the domain (e.g. vessels holding a substrate  */
/* at a fixed value): node i holds substrate sub[i] of voxel vox[i]    */
/* (x + nx (y + ny z)) at val[i].  Nodes are applied wherever the      */
/* Dirichlet shell is, right after it: before the x-solve and after    */
/* every solve; in index order, so of two nodes on one voxel and       */
/* substrate the later one holds.  Sources follow as before.           */
/* ------------------------------------------------------------------ */
void oracle_apply_nodes(int nx, int ny, int nz, int64_t n_nodes, const int64_t* vox,
                        const int* sub, const double* val, double* rho)
{
    const int64_t n_vox = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < n_nodes; ++i) rho[(int64_t)sub[i] * n_vox + vox[i]] = val[i];
}

int oracle_run_nodes(int nx, int ny, int nz, double dx, double dt, int n_sub,
                     const double* D, const double* lambda, const int* bc_kind,
                     const double* bc_value, int64_t n_cells, const double* pos,
                     const double* vol, const double* S, const double* U,
                     const double* rho_star, int64_t n_nodes, const int64_t* vox,
                     const int* sub, const double* val, int n_steps, int n_threads,
                     double* rho)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_sub < 1 || n_steps < 0) return 1;
    for (int64_t i = 0; i < n_nodes; ++i)
        if (vox[i] < 0 || vox[i] >= (int64_t)nx * ny * nz || sub[i] < 0 || sub[i] >= n_sub)
            return 2;
    for (int t = 0; t < n_steps; ++t) {
        oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, rho);
        oracle_apply_nodes(nx, ny, nz, n_nodes, vox, sub, val, rho);
        for (int axis = 0; axis < 3; ++axis) {
            oracle_axis_solve(axis, nx, ny, nz, n_sub, dx, dt, D, lambda, rho, n_threads);
            oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, rho);
            oracle_apply_nodes(nx, ny, nz, n_nodes, vox, sub, val, rho);
        }
        oracle_apply_sources(nx, ny, nz, n_sub, dx, dt, n_cells, pos, vol, S, U,
                             rho_star, rho);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Reverse mode of oracle_run: the literal adjoint of every operation  */
/* of every step, taken in reverse.                                     */
/*                                                                      */
/*  - sources: per voxel the cells were applied in ascending index;     */
/*    the reverse visits them in descending index.  For                 */
/*    f = (rho + a) / (1 + b):  df/drho = df/da = 1/(1+b),              */
/*    df/db = -f/(1+b);  a = w S rho*, b = w (S + U), w = dt V/V_vox.   */
/*  - Dirichlet: the shell of a Dirichlet substrate no longer depends   */
/*    on its input, so its adjoint is zeroed.                            */
/*  - Dirichlet nodes (oracle_adjoint_ext): likewise, a node's adjoint  */
/*    is zeroed after the shell's.                                       */
/*  - axis solve y = A^{-1} x: A is symmetric, so g_x = A^{-1} g_y, and */
/*    dL/dtheta -= <g_x, (dA/dtheta) y> with dA/dlambda = dt/3 I (dt/2   */
/*    in the 2-D variant, oracle_adjoint_ext with dims 2) and            */
/*    dA/dD = dt/dx^2 L, L the zero-flux line Laplacian (1 at both ends, */
/*    2 inside, -1 off the diagonal; 0 for a line of length 1).          */
/* The forward is recomputed from the initial field; the state at the   */
/* start of every `checkpoint_every`-th step is stored and each segment  */
/* is replayed step by step (replay is bit-identical to the first run).  */
/*                                                                      */
/* Inputs: rho0 (initial field), g_final = dL/d rho_final.              */
/* Outputs: dD[n_sub], dlambda[n_sub], dS[n_cells*n_sub],               */
/* dU[n_cells*n_sub] (accumulated from zero), g0 = dL/d rho0 (may be    */
/* NULL), rho_final (may be NULL).                                       */
/* ------------------------------------------------------------------ */

/* (L y) along one axis for every line of one substrate block. */
static double axis_laplacian_dot(int axis, int nx, int ny, int nz,
                                 const double* g, const double* y)
{
    int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
    int64_t stride = axis == 0 ? 1 : (axis == 1 ? (int64_t)nx : (int64_t)nx * ny);
    double acc = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int x = 0; x < nx; ++x) {
                int i = axis == 0 ? x : (axis == 1 ? yy : z);
                int64_t idx = ((int64_t)z * ny + yy) * (int64_t)nx + x;
                double ly = 0.0;
                if (n_axis > 1) {
                    if (i > 0) ly += y[idx] - y[idx - stride];
                    if (i < n_axis - 1) ly += y[idx] - y[idx + stride];
                }
                acc += g[idx] * ly;
            }
    return acc;
}

static double block_dot(int64_t n, const double* a, const double* b)
{
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += a[i] * b[i];
    return acc;
}

/* One step of the 3-D step with Dirichlet nodes (the step of
 * oracle_run_nodes; none: oracle_step's) or of the 2-D variant (dims 2, the
 * step of oracle_run_2d), in place. */
static void step_any(int dims, int nx, int ny, int nz, double dx, double dt, int n_sub,
                     const double* D, const double* lambda, const int* bc_kind,
                     const double* bc_value, int64_t n_cells, const double* pos,
                     const double* vol, const double* S, const double* U,
                     const double* rho_star, int64_t n_nodes, const int64_t* vox,
                     const int* sub, const double* val, double* rho, int n_threads)
{
    if (dims == 2) {
        oracle_apply_dirichlet_2d(nx, ny, n_sub, bc_kind, bc_value, rho);
        for (int axis = 0; axis < 2; ++axis) {
            oracle_axis_solve_2d(axis, nx, ny, n_sub, dx, dt, D, lambda, rho);
            oracle_apply_dirichlet_2d(nx, ny, n_sub, bc_kind, bc_value, rho);
        }
    } else {
        oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, rho);
        oracle_apply_nodes(nx, ny, nz, n_nodes, vox, sub, val, rho);
        for (int axis = 0; axis < 3; ++axis) {
            oracle_axis_solve(axis, nx, ny, nz, n_sub, dx, dt, D, lambda, rho, n_threads);
            oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, rho);
            oracle_apply_nodes(nx, ny, nz, n_nodes, vox, sub, val, rho);
        }
    }
    oracle_apply_sources(nx, ny, nz, n_sub, dx, dt, n_cells, pos, vol, S, U, rho_star, rho);
}

/* The 2-D shell (the four edges x = 0, nx-1, y = 0, ny-1) of a Dirichlet
 * substrate no longer depends on its input: its adjoint is zeroed. */
static void project_dirichlet_adjoint_2d(int nx, int ny, int n_sub, const int* bc_kind,
                                         double* g)
{
    for (int s = 0; s < n_sub; ++s) {
        if (bc_kind[s] != 1) continue;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)
                    g[((int64_t)s * ny + y) * nx + x] = 0.0;
    }
}

/* A Dirichlet node's value no longer depends on its input: its adjoint
 * is zeroed. */
static void project_nodes_adjoint(int nx, int ny, int nz, int64_t n_nodes, const int64_t* vox,
                                  const int* sub, double* g)
{
    const int64_t n_vox = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < n_nodes; ++i) g[(int64_t)sub[i] * n_vox + vox[i]] = 0.0;
}

static int adjoint_any(int dims, int nx, int ny, int nz, double dx, double dt, int n_sub,
                       const double* D, const double* lambda, const int* bc_kind,
                       const double* bc_value, int64_t n_cells, const double* pos,
                       const double* vol, const double* S, const double* U,
                       const double* rho_star, int64_t n_nodes, const int64_t* vox,
                       const int* sub, const double* val, int n_steps, int checkpoint_every,
                       int n_threads, const double* rho0, const double* g_final,
                       double* dD, double* dlambda, double* dS, double* dU,
                       double* g0, double* rho_final);

int oracle_adjoint(int nx, int ny, int nz, double dx, double dt, int n_sub,
                   const double* D, const double* lambda, const int* bc_kind,
                   const double* bc_value, int64_t n_cells, const double* pos,
                   const double* vol, const double* S, const double* U,
                   const double* rho_star, int n_steps, int checkpoint_every,
                   int n_threads, const double* rho0, const double* g_final,
                   double* dD, double* dlambda, double* dS, double* dU,
                   double* g0, double* rho_final)
{
    return adjoint_any(3, nx, ny, nz, dx, dt, n_sub, D, lambda, bc_kind, bc_value, n_cells,
                       pos, vol, S, U, rho_star, 0, NULL, NULL, NULL, n_steps,
                       checkpoint_every, n_threads, rho0, g_final, dD, dlambda, dS, dU, g0,
                       rho_final);
}

/* The adjoint of the 2-D variant (dims 2: nz = 1, x- and y-solves with
 * decay share lambda dt / 2, the four-edge shell) or of the 3-D step with
 * Dirichlet nodes (dims 3; each node projection's adjoint zeroes the node's
 * entry, right after the shell's).  Arguments as oracle_adjoint, with the
 * nodes as in oracle_run_nodes (none for dims 2). */
int oracle_adjoint_ext(int dims, int nx, int ny, int nz, double dx, double dt, int n_sub,
                       const double* D, const double* lambda, const int* bc_kind,
                       const double* bc_value, int64_t n_cells, const double* pos,
                       const double* vol, const double* S, const double* U,
                       const double* rho_star, int64_t n_nodes, const int64_t* vox,
                       const int* sub, const double* val, int n_steps, int checkpoint_every,
                       int n_threads, const double* rho0, const double* g_final,
                       double* dD, double* dlambda, double* dS, double* dU,
                       double* g0, double* rho_final)
{
    if (dims != 2 && dims != 3) return 1;
    if (dims == 2 && (nz != 1 || n_nodes != 0)) return 1;
    for (int64_t i = 0; i < n_nodes; ++i)
        if (vox[i] < 0 || vox[i] >= (int64_t)nx * ny * nz || sub[i] < 0 || sub[i] >= n_sub)
            return 2;
    return adjoint_any(dims, nx, ny, nz, dx, dt, n_sub, D, lambda, bc_kind, bc_value, n_cells,
                       pos, vol, S, U, rho_star, n_nodes, vox, sub, val, n_steps,
                       checkpoint_every, n_threads, rho0, g_final, dD, dlambda, dS, dU, g0,
                       rho_final);
}

static int adjoint_any(int dims, int nx, int ny, int nz, double dx, double dt, int n_sub,
                       const double* D, const double* lambda, const int* bc_kind,
                       const double* bc_value, int64_t n_cells, const double* pos,
                       const double* vol, const double* S, const double* U,
                       const double* rho_star, int64_t n_nodes, const int64_t* vox,
                       const int* sub, const double* val, int n_steps, int checkpoint_every,
                       int n_threads, const double* rho0, const double* g_final,
                       double* dD, double* dlambda, double* dS, double* dU,
                       double* g0, double* rho_final)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_sub < 1 || n_steps < 0) return 1;
    if (checkpoint_every < 1) checkpoint_every = 1;
    int64_t n_vox = (int64_t)nx * ny * nz;
    int64_t n_field = n_vox * n_sub;
    size_t fbytes = sizeof(double) * (size_t)n_field;
    int n_ckpt = (n_steps + checkpoint_every - 1) / checkpoint_every;
    double* ckpt = (double*)malloc(fbytes * (size_t)(n_ckpt > 0 ? n_ckpt : 1));
    double* cur = (double*)malloc(fbytes);
    double* g = (double*)malloc(fbytes);
    /* states inside one step: after Dirichlet prologue, after each raw
     * axis solve (before its Dirichlet), before the sources */
    double* seg = (double*)malloc(fbytes * (size_t)checkpoint_every);
    double* st_solve[3];
    double* st_pre_src = (double*)malloc(fbytes);
    for (int a = 0; a < 3; ++a) st_solve[a] = (double*)malloc(fbytes);
    double* tmp = (double*)malloc(fbytes);
    if (!ckpt || !cur || !g || !seg || !st_pre_src || !st_solve[0] ||
        !st_solve[1] || !st_solve[2] || !tmp) return 2;

    memcpy(cur, rho0, fbytes);
    for (int t = 0; t < n_steps; ++t) {
        if (t % checkpoint_every == 0)
            memcpy(ckpt + (size_t)(t / checkpoint_every) * n_field, cur, fbytes);
        step_any(dims, nx, ny, nz, dx, dt, n_sub, D, lambda, bc_kind, bc_value, n_cells, pos,
                 vol, S, U, rho_star, n_nodes, vox, sub, val, cur, n_threads);
    }
    if (rho_final) memcpy(rho_final, cur, fbytes);

    for (int s = 0; s < n_sub; ++s) { dD[s] = 0.0; dlambda[s] = 0.0; }
    for (int64_t i = 0; i < n_cells * n_sub; ++i) { dS[i] = 0.0; dU[i] = 0.0; }
    memcpy(g, g_final, fbytes);

    double v_vox = dx * dx * dx;
    int64_t* cell_vox = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_cells > 0 ? n_cells : 1));
    double* before = (double*)malloc(sizeof(double) * (size_t)(n_cells * n_sub > 0 ? n_cells * n_sub : 1));
    for (int64_t i = 0; i < n_cells; ++i)
        cell_vox[i] = oracle_cell_voxel(nx, ny, nz, dx, pos + 3 * i);

    for (int k = n_ckpt - 1; k >= 0; --k) {
        int t0 = k * checkpoint_every;
        int t1 = t0 + checkpoint_every < n_steps ? t0 + checkpoint_every : n_steps;
        /* replay the segment, keeping each step's input state */
        memcpy(cur, ckpt + (size_t)k * n_field, fbytes);
        for (int t = t0; t < t1; ++t) {
            memcpy(seg + (size_t)(t - t0) * n_field, cur, fbytes);
            step_any(dims, nx, ny, nz, dx, dt, n_sub, D, lambda, bc_kind, bc_value, n_cells,
                     pos, vol, S, U, rho_star, n_nodes, vox, sub, val, cur, n_threads);
        }
        for (int t = t1 - 1; t >= t0; --t) {
            /* recompute the inner states of step t */
            memcpy(tmp, seg + (size_t)(t - t0) * n_field, fbytes);
            if (dims == 2) {
                oracle_apply_dirichlet_2d(nx, ny, n_sub, bc_kind, bc_value, tmp);
            } else {
                oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, tmp);
                oracle_apply_nodes(nx, ny, nz, n_nodes, vox, sub, val, tmp);
            }
            for (int a = 0; a < dims; ++a) {
                if (dims == 2)
                    oracle_axis_solve_2d(a, nx, ny, n_sub, dx, dt, D, lambda, tmp);
                else
                    oracle_axis_solve(a, nx, ny, nz, n_sub, dx, dt, D, lambda, tmp, n_threads);
                memcpy(st_solve[a], tmp, fbytes);
                if (dims == 2) {
                    oracle_apply_dirichlet_2d(nx, ny, n_sub, bc_kind, bc_value, tmp);
                } else {
                    oracle_apply_dirichlet(nx, ny, nz, n_sub, bc_kind, bc_value, tmp);
                    oracle_apply_nodes(nx, ny, nz, n_nodes, vox, sub, val, tmp);
                }
            }
            memcpy(st_pre_src, tmp, fbytes);
            /* forward through the sources, remembering each cell's input */
            for (int64_t i = 0; i < n_cells; ++i) {
                double w = dt * (vol[i] / v_vox);
                for (int s = 0; s < n_sub; ++s) {
                    double a = w * S[i * n_sub + s] * rho_star[i * n_sub + s];
                    double b = w * (S[i * n_sub + s] + U[i * n_sub + s]);
                    double* r = tmp + (int64_t)s * n_vox + cell_vox[i];
                    before[i * n_sub + s] = *r;
                    *r = (*r + a) / (1.0 + b);
                }
            }
            /* adjoint of the sources, descending cell index */
            for (int64_t i = n_cells - 1; i >= 0; --i) {
                double w = dt * (vol[i] / v_vox);
                for (int s = 0; s < n_sub; ++s) {
                    double a = w * S[i * n_sub + s] * rho_star[i * n_sub + s];
                    double b = w * (S[i * n_sub + s] + U[i * n_sub + s]);
                    double f = (before[i * n_sub + s] + a) / (1.0 + b);
                    double* gv = g + (int64_t)s * n_vox + cell_vox[i];
                    double ga = *gv / (1.0 + b);
                    double gb = -(*gv) * f / (1.0 + b);
                    dS[i * n_sub + s] += ga * w * rho_star[i * n_sub + s] + gb * w;
                    dU[i * n_sub + s] += gb * w;
                    *gv = *gv / (1.0 + b);
                }
            }
            /* adjoint of the z, y, x solves (y, x in 2-D), each preceded by
             * its Dirichlet (and nodes); each axis takes lambda dt / dims */
            for (int a = dims - 1; a >= 0; --a) {
                if (dims == 2) {
                    project_dirichlet_adjoint_2d(nx, ny, n_sub, bc_kind, g);
                    oracle_axis_solve_2d(a, nx, ny, n_sub, dx, dt, D, lambda, g);
                } else {
                    project_dirichlet_adjoint(nx, ny, nz, n_sub, bc_kind, g);
                    project_nodes_adjoint(nx, ny, nz, n_nodes, vox, sub, g);
                    oracle_axis_solve(a, nx, ny, nz, n_sub, dx, dt, D, lambda, g, n_threads);
                }
                for (int s = 0; s < n_sub; ++s) {
                    const double* gs = g + (int64_t)s * n_vox;
                    const double* ys = st_solve[a] + (int64_t)s * n_vox;
                    dlambda[s] -= (dt / (double)dims) * block_dot(n_vox, gs, ys);
                    dD[s] -= (dt / (dx * dx)) * axis_laplacian_dot(a, nx, ny, nz, gs, ys);
                }
            }
            if (dims == 2) {
                project_dirichlet_adjoint_2d(nx, ny, n_sub, bc_kind, g);
            } else {
                project_dirichlet_adjoint(nx, ny, nz, n_sub, bc_kind, g);
                project_nodes_adjoint(nx, ny, nz, n_nodes, vox, sub, g);
            }
        }
    }
    if (g0) memcpy(g0, g, fbytes);
    free(ckpt); free(cur); free(g); free(seg); free(st_pre_src);
    for (int a = 0; a < 3; ++a) free(st_solve[a]);
    free(tmp); free(cell_vox); free(before);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
