/*
 * FP64 CPU oracle for the fused periodic 2D Poisson relaxation sweep.
 *
 * TEST INFRASTRUCTURE ONLY. It is called by the tests, by the smoke check and
 * by the CPU-baseline leg of the benchmark; the product path never links it.
 * It shares no code, header or constant with the CUDA library.
 *
 * What it computes (ProtoX, Sec. IV):
 *   - the model problem Delta phi = rho on a periodic, cell-centred grid with
 *     spacing h, discretised by the 5-point Laplacian (Sec. IV, "2D Poisson
 *     equation"; taps [0,1,0; 1,-4,1; 0,1,0] of the OL Laplace rule);
 *   - the Jacobi step (Eq. "jacobi"), generalised to a weight omega:
 *       phi' = phi + w*s - lam*rho,  s = unscaled tap sum,
 *       w = omega/4, lam = omega*h^2/4   (OL rule Jacobi = (1, w, -lambda) x I);
 *     the paper's own lambda = h^2/(4D) is the case omega = 1/D = 1/2;
 *   - the max-norm of the residual of the INPUT state of each sweep,
 *       R = max |s/h^2 - rho|            (OL rule ||.||_inf = Max o pw|x| o (0, 1/a^2, -1));
 *   - one layer of periodic ghost cells (Sec. III, "Proto": periodic boundary
 *     conditions; Sec. IV: n x n box stored with m = n + 2 including ghosts).
 *
 * Evaluation order is fixed and the file is compiled with -ffp-contract=off,
 * so every function here is bitwise reproducible:
 *   s   = ((pW + pE) + (pS + pN)) - 4.0*pC
 *   phi'= (pC + w*s) - lam*rho
 *   r   = fabs(ih2*s - rho),  ih2 = 1/(h*h)
 * The unfused mode (Sec. IV, Fig. "Proto": Laplacian into a temporary, an
 * in-place Jacobi pass, then a separate residual pass) uses the same per-point
 * expressions, so fused and unfused agree bitwise; the unfused residual of
 * iteration n is the fused residual reported by sweep n+1.
 *
 * Arrays are row-major, x fastest: a[j*ld + i], i in [0,nx), j in [0,ny).
 * Parity pins: every function here is checked in the CPU test-suite against
 * closed-form eigenmodes, a dense-matrix Jacobi iteration, library routines
 * (eigvalsh, FFT solve) and invariants, never against itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Running max that keeps a NaN once one has been seen (a NaN residual must
 * surface as NaN, not be hidden by later finite values). */
static double maxnan(double R, double r) {
  return (r > R || r != r) ? r : R;
}

static int64_t wrapi(int64_t i, int64_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

/* Periodic ghost fill of a ghosted array: (ny+2) rows of pitch ld >= nx+2,
 * interior cell (i,j) at g[(j+1)*ld + (i+1)]. Corners are filled too
 * (the 5-point stencil never reads them). Sec. III "Proto", Sec. IV layout. */
void oracle_fill_ghosts(int nx, int ny, int64_t ld, double* g) {
  for (int j = 1; j <= ny; ++j) {
    g[(int64_t)j * ld + 0] = g[(int64_t)j * ld + nx];
    g[(int64_t)j * ld + nx + 1] = g[(int64_t)j * ld + 1];
  }
  memcpy(g, g + (int64_t)ny * ld, sizeof(double) * (size_t)(nx + 2));
  memcpy(g + (int64_t)(ny + 1) * ld, g + ld, sizeof(double) * (size_t)(nx + 2));
}

/* Unscaled 5-point tap sum at (i,j) of an unghosted periodic array. */
static double taps(int nx, int ny, int64_t ld, const double* p, int i, int j) {
  int64_t jm = wrapi(j - 1, ny), jp = wrapi(j + 1, ny);
  int64_t im = wrapi(i - 1, nx), ip = wrapi(i + 1, nx);
  double pC = p[(int64_t)j * ld + i];
  double pW = p[(int64_t)j * ld + im], pE = p[(int64_t)j * ld + ip];
  double pS = p[jm * ld + i], pN = p[jp * ld + i];
  return ((pW + pE) + (pS + pN)) - 4.0 * pC;
}

/* out = L phi = s/h^2 (the Laplace operator of the OL spec, scaled by 1/a^2
 * with a = h). Periodic, unghosted, pitch ld for both arrays. */
void oracle_apply_stencil(int nx, int ny, int64_t ld, double h,
                          const double* phi, double* out) {
  double ih2 = 1.0 / (h * h);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      out[(int64_t)j * ld + i] = ih2 * taps(nx, ny, ld, phi, i, j);
}

/* max |rho - L phi| and max |rho| over all cells (Sec. IV step 3: max-norm
 * convergence check). Either output may be NULL. */
void oracle_residual_norm(int nx, int ny, int64_t ld, double h,
                          const double* phi, const double* rho,
                          double* rnorm, double* rho_norm) {
  double ih2 = 1.0 / (h * h), R = 0.0, P = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double s = taps(nx, ny, ld, phi, i, j);
      double rv = rho[(int64_t)j * ld + i];
      double r = fabs(ih2 * s - rv);
      R = maxnan(R, r);
      double a = fabs(rv);
      P = maxnan(P, a);
    }
  if (rnorm) *rnorm = R;
  if (rho_norm) *rho_norm = P;
}

/* One fused sweep (Laplace, Jacobi and max-norm in one loop over the cells,
 * the Sigma-OL merged form of Sec. IV). Reads phi, writes phinew (must not
 * alias phi), returns the max-norm residual of the input state phi. */
double oracle_sweep(int nx, int ny, int64_t ld, double h, double omega,
                    const double* phi, const double* rho, double* phinew) {
  double ih2 = 1.0 / (h * h);
  double w = omega / 4.0, lam = omega * h * h / 4.0;
  double R = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int64_t c = (int64_t)j * ld + i;
      double s = taps(nx, ny, ld, phi, i, j);
      double rv = rho[c];
      phinew[c] = (phi[c] + w * s) - lam * rv;
      double r = fabs(ih2 * s - rv);
      R = maxnan(R, r);
    }
  return R;
}

/* n fused sweeps from phi0 (not modified) into phi_out (contiguous, ld = nx).
 * Reports resid[k] = ||rho - L phi^(k*every)||_inf for every state index that
 * is a multiple of `every` and < nsweeps (computed by the sweep that reads
 * that state). resid may be NULL or every <= 0 for no reports.
 * Returns 0, or -1 on allocation failure. */
int oracle_relax_n(int nx, int ny, double h, double omega, const double* phi0,
                   const double* rho, int nsweeps, int every, double* phi_out,
                   double* resid) {
  size_t n = (size_t)nx * (size_t)ny;
  double* a = (double*)malloc(n * sizeof(double));
  double* b = (double*)malloc(n * sizeof(double));
  if (!a || !b) { free(a); free(b); return -1; }
  memcpy(a, phi0, n * sizeof(double));
  for (int s = 0; s < nsweeps; ++s) {
    double R = oracle_sweep(nx, ny, nx, h, omega, a, rho, b);
    if (resid && every > 0 && s % every == 0) resid[s / every] = R;
    double* t = a; a = b; b = t;
  }
  memcpy(phi_out, a, n * sizeof(double));
  free(a); free(b);
  return 0;
}

/* The unfused program of Fig. "Proto", on ghosted storage (m = n+2 style):
 * per iteration (1) ghost exchange, (2) temp = Laplacian taps of phi over the
 * box, (3) Jacobi update of phi in place from temp and rho, (4) ghost exchange
 * and a separate max-norm pass over the updated phi.
 * g: (ny+2) x (nx+2) ghosted phi, updated in place; rho: ny x nx unghosted.
 * resid[it] = residual of the state after iteration it (may be NULL). */
int oracle_relax_unfused(int nx, int ny, double h, double omega, double* g,
                         const double* rho, int iters, double* resid) {
  int64_t ld = nx + 2;
  double ih2 = 1.0 / (h * h);
  double w = omega / 4.0, lam = omega * h * h / 4.0;
  double* temp = (double*)malloc((size_t)nx * (size_t)ny * sizeof(double));
  if (!temp) return -1;
  for (int it = 0; it < iters; ++it) {
    oracle_fill_ghosts(nx, ny, ld, g);
    for (int j = 0; j < ny; ++j)        /* pass 1: temp = stencil(phi) */
      for (int i = 0; i < nx; ++i) {
        const double* p = g + (int64_t)(j + 1) * ld + (i + 1);
        temp[(int64_t)j * nx + i] = ((p[-1] + p[1]) + (p[-ld] + p[ld])) - 4.0 * p[0];
      }
    for (int j = 0; j < ny; ++j)        /* pass 2: forallInPlace(jacobi) */
      for (int i = 0; i < nx; ++i) {
        double* p = g + (int64_t)(j + 1) * ld + (i + 1);
        *p = (*p + w * temp[(int64_t)j * nx + i]) - lam * rho[(int64_t)j * nx + i];
      }
    oracle_fill_ghosts(nx, ny, ld, g);  /* pass 3: max residual */
    double R = 0.0;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double* p = g + (int64_t)(j + 1) * ld + (i + 1);
        double s = ((p[-1] + p[1]) + (p[-ld] + p[ld])) - 4.0 * p[0];
        double r = fabs(ih2 * s - rho[(int64_t)j * nx + i]);
        R = maxnan(R, r);
      }
    if (resid) resid[it] = R;
  }
  free(temp);
  return 0;
}

/* Fused sweeps on ghosted storage: X and Y are (ny+2) x (nx+2) arrays, ghosts
 * of X are filled before each sweep, rho is unghosted. Same arithmetic as
 * oracle_sweep. Result ends in X after an even count; returns the array that
 * holds the final state (0 = X, 1 = Y). */
int oracle_relax_ghosted(int nx, int ny, double h, double omega, double* X,
                         double* Y, const double* rho, int nsweeps, double* resid) {
  int64_t ld = nx + 2;
  double ih2 = 1.0 / (h * h);
  double w = omega / 4.0, lam = omega * h * h / 4.0;
  double *a = X, *b = Y;
  for (int s = 0; s < nsweeps; ++s) {
    oracle_fill_ghosts(nx, ny, ld, a);
    double R = 0.0;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = (int64_t)(j + 1) * ld + (i + 1);
        const double* p = a + c;
        double s5 = ((p[-1] + p[1]) + (p[-ld] + p[ld])) - 4.0 * p[0];
        double rv = rho[(int64_t)j * nx + i];
        b[c] = (p[0] + w * s5) - lam * rv;
        double r = fabs(ih2 * s5 - rv);
        R = maxnan(R, r);
      }
    if (resid) resid[s] = R;
    double* t = a; a = b; b = t;
  }
  return a == X ? 0 : 1;
}

/* OpenMP fused sweeps (rows split over threads, max combined by an OpenMP
 * max-reduction). Used only to time the CPU baseline on all host cores; the
 * arithmetic per cell is that of oracle_sweep. Returns threads used. */
int oracle_relax_n_omp(int nx, int ny, double h, double omega, double* a,
                       double* b, const double* rho, int nsweeps, int nthreads,
                       double* last_resid) {
  double ih2 = 1.0 / (h * h);
  double w = omega / 4.0, lam = omega * h * h / 4.0;
  int used = 1;
  double R = 0.0;
  for (int s = 0; s < nsweeps; ++s) {
    R = 0.0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) reduction(max : R) schedule(static)
#endif
    for (int j = 0; j < ny; ++j) {
#ifdef _OPENMP
      if (j == 0) used = omp_get_num_threads();
#endif
      for (int i = 0; i < nx; ++i) {
        int64_t c = (int64_t)j * nx + i;
        double sv = taps(nx, ny, nx, a, i, j);
        double rv = rho[c];
        b[c] = (a[c] + w * sv) - lam * rv;
        double r = fabs(ih2 * sv - rv);
        if (r > R) R = r;
      }
    }
    double* t = a; a = b; b = t;
  }
  if (last_resid) *last_resid = R;
  (void)nthreads;
  return used;
}

/* Red-black SOR: the relaxation the paper names as the smoother of Proto's
 * multigrid (Sec. VI, future work), in its standard definition. One sweep
 * updates IN PLACE first every red cell ((i + j) even), then every black cell
 * ((i + j) odd), each with the Jacobi per-point update of oracle_sweep,
 *     phi[i,j] <- (phi + w*s) - lam*rho,  w = omega/4, lam = omega*h^2/4,
 * where s is the tap sum of the CURRENT array: during the red half all
 * neighbours (black) are still old, during the black half all neighbours
 * (red) are already new. omega = 1 is red-black Gauss-Seidel. nx and ny must
 * be even, so that the colouring agrees across the periodic wrap. The
 * residual reported for a sweep is that of its INPUT state, over all cells,
 * in the expressions of oracle_sweep.
 * Returns 0, -1 on allocation failure, -2 for an odd extent. */
int oracle_rbsor_n(int nx, int ny, double h, double omega, const double* phi0,
                   const double* rho, int nsweeps, int every, double* phi_out,
                   double* resid) {
  if (nx % 2 != 0 || ny % 2 != 0) return -2;
  size_t n = (size_t)nx * (size_t)ny;
  double* a = (double*)malloc(n * sizeof(double));
  if (!a) return -1;
  memcpy(a, phi0, n * sizeof(double));
  double ih2 = 1.0 / (h * h);
  double w = omega / 4.0, lam = omega * h * h / 4.0;
  for (int s = 0; s < nsweeps; ++s) {
    if (resid && every > 0 && s % every == 0) {
      double R = 0.0;
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          R = maxnan(R, fabs(ih2 * taps(nx, ny, nx, a, i, j) - rho[(int64_t)j * nx + i]));
      resid[s / every] = R;
    }
    for (int colour = 0; colour < 2; ++colour)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          if (((i + j) & 1) != colour) continue;
          int64_t c = (int64_t)j * nx + i;
          double sv = taps(nx, ny, nx, a, i, j);
          a[c] = (a[c] + w * sv) - lam * rho[c];
        }
  }
  memcpy(phi_out, a, n * sizeof(double));
  free(a);
  return 0;
}

/* ---------------------------------------------------------------------------
 * 3D periodic Poisson, 7-point stencil (the paper's Eq. "jacobi" in D = 3
 * dimensions: lambda = h^2 / (4 D) is the omega = 1/2 case of the weight
 * omega h^2 / (2 D) = omega h^2 / 6). Arrays are contiguous [z][y][x].
 * Unscaled tap sum s = ((W + E) + (S + N)) + (B + T) - 6 C. */
static double taps3(int nx, int ny, int nz, const double* p, int i, int j, int k) {
  int64_t pl = (int64_t)nx * ny;
  int64_t im = wrapi(i - 1, nx), ip = wrapi(i + 1, nx);
  int64_t jm = wrapi(j - 1, ny), jp = wrapi(j + 1, ny);
  int64_t km = wrapi(k - 1, nz), kp = wrapi(k + 1, nz);
  int64_t row = (int64_t)k * pl + (int64_t)j * nx;
  double pC = p[row + i];
  double pW = p[row + im], pE = p[row + ip];
  double pS = p[(int64_t)k * pl + jm * nx + i], pN = p[(int64_t)k * pl + jp * nx + i];
  double pB = p[km * pl + (int64_t)j * nx + i], pT = p[kp * pl + (int64_t)j * nx + i];
  return (((pW + pE) + (pS + pN)) + (pB + pT)) - 6.0 * pC;
}

/* One fused 3D sweep: phinew = (C + w s) - lam rho with w = omega / 6,
 * lam = omega h^2 / 6; returns ||s/h^2 - rho||_inf of the input state. */
double oracle_sweep3(int nx, int ny, int nz, double h, double omega, const double* phi,
                     const double* rho, double* phinew) {
  double ih2 = 1.0 / (h * h);
  double w = omega / 6.0, lam = omega * h * h / 6.0;
  double R = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = ((int64_t)k * ny + j) * nx + i;
        double s = taps3(nx, ny, nz, phi, i, j, k);
        double rv = rho[c];
        phinew[c] = (phi[c] + w * s) - lam * rv;
        double r = fabs(ih2 * s - rv);
        R = maxnan(R, r);
      }
  return R;
}

/* n fused 3D sweeps from phi0 into phi_out; reports as oracle_relax_n.
 * Returns 0, or -1 on allocation failure. */
int oracle_relax3_n(int nx, int ny, int nz, double h, double omega, const double* phi0,
                    const double* rho, int nsweeps, int every, double* phi_out,
                    double* resid) {
  size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
  double* a = (double*)malloc(n * sizeof(double));
  double* b = (double*)malloc(n * sizeof(double));
  if (!a || !b) { free(a); free(b); return -1; }
  memcpy(a, phi0, n * sizeof(double));
  for (int s = 0; s < nsweeps; ++s) {
    double R = oracle_sweep3(nx, ny, nz, h, omega, a, rho, b);
    if (resid && every > 0 && s % every == 0) resid[s / every] = R;
    double* t = a; a = b; b = t;
  }
  memcpy(phi_out, a, n * sizeof(double));
  free(a); free(b);
  return 0;
}
