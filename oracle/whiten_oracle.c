/*
 * FP64 CPU oracle for the recursive clutter-whitening preprocessor of
 * H. L. Kennedy, "Parallel software implementation of recursive
 * multidimensional digital filters for point-target detection in cluttered
 * infrared scenes" (arXiv:1408.3526).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code,
 * header, table or constant with the CUDA path of the product.
 *
 * Plain, slow, obviously correct: every step follows the paper's order and
 * notation in double precision (no fast-math, no FMA contraction), with the
 * readings below where the paper is silent or garbled:
 *   - temporal order Mz is the number of temporal bins/observer states; even
 *     Mz is allowed, bins kz = -((Mz-1)/2) .. Mz/2 (Sec. 2 uses odd M = 2K+1)
 *   - frame borders: reads outside the frame are clamped to the edge pixel
 *   - history before frame 0 is zero (observer state starts at 0), smoother
 *     state starts at 0
 *   - "spatial components with k = 0 are omitted": the bins kx = ky = 0 are
 *     zeroed (all kz) before the Hann window; the PEF keeps them
 *   - Hann window: centred w(m) = 1/2 + 1/2 cos(2 pi (m - D)/M), D = (M-1)/2,
 *     applied as the circular 3-tap convolution it induces in k
 *   - Eq. (8h) is read with Delta_z in place of Delta_x
 *   - Dirichlet kernel at integer arguments takes its limit value
 *   - argmax ties go to the lowest flat grid index iy*L + ix
 *   - output delay m'_z = floor((Mz-1)/2) unless given
 *
 * Layout: frames float32 [T][H][W] row-major, x = column.  Spectrum bins per
 * pixel [iz][iy][ix] with kx = ix - K, ky = iy - K, kz = iz + kzlo,
 * kzlo = -((Mz-1)/2).  Velocity grid value i -> -vmax + i*vstep, flat index
 * iy*L + ix.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------------- */
/* Dirichlet kernel of order W, Eq. (3): D_W(w) = sin(pi W w)/(W sin(pi w)).
 * Written about the nearest integer j (w = j + d, |d| <= 1/2):
 *   D_W(j + d) = (-1)^(j (W-1)) sin(pi W d)/(W sin(pi d)),
 * which is exact and takes the limit value (-1)^(j(W-1)) at d = 0.       */
double orc_dirichlet(int W, double w)
{
    double j = nearbyint(w);
    double d = w - j;
    long long ji = (long long)j;
    double sgn = ((ji * (long long)(W - 1)) % 2 == 0) ? 1.0 : -1.0;
    if (fabs(d) < 1e-9) {
        /* series: sin(pi W d)/(W sin(pi d)) = 1 - (pi d)^2 (W^2 - 1)/6 + O(d^4) */
        double pd = PI * d;
        return sgn * (1.0 - pd * pd * ((double)W * W - 1.0) / 6.0);
    }
    return sgn * sin(PI * W * d) / (W * sin(PI * d));
}

/* ---------------------------------------------------------------------- */
/* Sliding DFT of one line (Sec. 1: a comb filter cascaded with a resonator):
 *   c(n) = e(n) - e(n - M),  Y(n) = exp(j 2 pi k / M) Y(n-1) + c(n),
 * with e = 0 before the line and Y(-1) = 0, so that once n >= M-1,
 *   Y(n) = sum_{m=0}^{M-1} exp(j 2 pi k m / M) e(n - m)     (Eq. (6), one axis). */
void orc_sdft_line(const cplx *e, int len, int M, int k, cplx *out)
{
    cplx w = cexp(I * 2.0 * PI * (double)k / (double)M);
    cplx y = 0.0;
    for (int n = 0; n < len; ++n) {
        cplx c = e[n] - (n >= M ? e[n - M] : 0.0);
        y = w * y + c;
        out[n] = y;
    }
}

/* ---------------------------------------------------------------------- */
/* Deadbeat observer bank over time (Sec. 1, [12],[14]): Mz integrator states
 * s_k rotating at lambda_k = exp(j 2 pi kz / Mz); the prediction is their sum
 * and the error e = u - yhat is fed back equally to every state:
 *   a_k = s_k + e / Mz   (a-posteriori state)
 *   s_k <- lambda_k a_k  (prediction for the next frame).
 * All closed-loop poles sit at z = 0, so after Mz frames a_k equals
 * (1/Mz) sum_{mz} u(n - mz) exp(j 2 pi kz mz / Mz) exactly, whatever the
 * initial state.  'a' receives the a-posteriori states (index iz). */
void orc_observer_step(cplx *s, int Mz, int kzlo, cplx u, cplx *a)
{
    cplx yhat = 0.0;
    for (int i = 0; i < Mz; ++i) yhat += s[i];
    cplx e = u - yhat;
    for (int i = 0; i < Mz; ++i) {
        double kz = (double)(i + kzlo);
        cplx lam = cexp(I * 2.0 * PI * kz / (double)Mz);
        a[i] = s[i] + e / (double)Mz;
        s[i] = lam * a[i];
    }
}

/* Run the observer over a sequence u[0..n) from initial state s0 (Mz
 * complex, may be NULL for zeros); a_out [n][Mz] a-posteriori states. */
void orc_observer_run(const double *u_re, const double *u_im, int n, int Mz,
                      const double *s0_re, const double *s0_im,
                      double *a_re, double *a_im)
{
    int kzlo = -((Mz - 1) / 2);
    cplx *s = (cplx *)calloc((size_t)Mz, sizeof(cplx));
    cplx *a = (cplx *)malloc((size_t)Mz * sizeof(cplx));
    if (s0_re)
        for (int i = 0; i < Mz; ++i) s[i] = s0_re[i] + I * s0_im[i];
    for (int t = 0; t < n; ++t) {
        orc_observer_step(s, Mz, kzlo, u_re[t] + I * u_im[t], a);
        for (int i = 0; i < Mz; ++i) {
            a_re[(size_t)t * Mz + i] = creal(a[i]);
            a_im[(size_t)t * Mz + i] = cimag(a[i]);
        }
    }
    free(s);
    free(a);
}

/* ---------------------------------------------------------------------- */
/* Frequency-sampling PEF design, Eq. (8a)-(8k), evaluated at the DFT bins
 * f = [k'x/M, k'y/M, k'z/Mz] (Sec. 2, after Eq. (8)):
 *   Q(f) = 1/sqrt(Mx My Mz) sum_{ky=-B}^{B} sum_{kx=-B}^{B} q(f)
 *   q    = bx by bz cx cy cz dx dy dz
 *   bx = exp(-j2pi kx/Mx (m'x - Dx)),   cx = exp(-j2pi fx Dx),
 *   by = exp(-j2pi ky/My (m'y - Dy)),   cy = exp(-j2pi fy Dy),
 *   bz = exp(+j2pi (vx kx/Mx + vy ky/My)(m'z - Dz)),  cz = exp(-j2pi fz Dz),
 *   dx = D_Mx(fx - kx/Mx),  dy = D_My(fy - ky/My),
 *   dz = D_Mz(fz + vx kx/Mx + vy ky/My),   D = (M-1)/2 per dimension.
 * Output H[iz][jy][jx] for k'x = jx - B, k'y = jy - B (|k'| <= B), all kz. */
void orc_pef_design(int M, int Mz, int B, int mpx, int mpy, int mpz,
                    double vx, double vy, double *h_re, double *h_im)
{
    int kzlo = -((Mz - 1) / 2);
    int W = 2 * B + 1;
    double Dx = (M - 1) / 2.0, Dy = (M - 1) / 2.0, Dz = (Mz - 1) / 2.0;
    double Mx = M, My = M, Mzd = Mz;
    double norm = 1.0 / sqrt(Mx * My * Mzd);
    /* the factors of Eq. (8b), tabulated over their own indices */
    cplx *bx = (cplx *)malloc(sizeof(cplx) * W), *by = (cplx *)malloc(sizeof(cplx) * W);
    cplx *cx = (cplx *)malloc(sizeof(cplx) * W), *cy = (cplx *)malloc(sizeof(cplx) * W);
    cplx *cz = (cplx *)malloc(sizeof(cplx) * Mz);
    cplx *bz = (cplx *)malloc(sizeof(cplx) * W * W);
    double *dx = (double *)malloc(sizeof(double) * W * W);   /* [jx][kx] */
    double *dy = (double *)malloc(sizeof(double) * W * W);   /* [jy][ky] */
    double *dz = (double *)malloc(sizeof(double) * Mz * W * W); /* [iz][ky][kx] */
    for (int k = -B; k <= B; ++k) {
        bx[k + B] = cexp(-I * 2.0 * PI * (k / Mx) * (mpx - Dx));       /* (8c) */
        by[k + B] = cexp(-I * 2.0 * PI * (k / My) * (mpy - Dy));       /* (8d) */
        cx[k + B] = cexp(-I * 2.0 * PI * (k / Mx) * Dx);               /* (8f), fx = k/Mx */
        cy[k + B] = cexp(-I * 2.0 * PI * (k / My) * Dy);               /* (8g) */
    }
    for (int iz = 0; iz < Mz; ++iz)
        cz[iz] = cexp(-I * 2.0 * PI * ((iz + kzlo) / Mzd) * Dz);       /* (8h), Delta_z */
    for (int j = -B; j <= B; ++j)
        for (int k = -B; k <= B; ++k) {
            dx[(j + B) * W + (k + B)] = orc_dirichlet(M, j / Mx - k / Mx);   /* (8i) */
            dy[(j + B) * W + (k + B)] = orc_dirichlet(M, j / My - k / My);   /* (8j) */
        }
    for (int ky = -B; ky <= B; ++ky)
        for (int kx = -B; kx <= B; ++kx) {
            double u = vx * kx / Mx + vy * ky / My;
            bz[(ky + B) * W + (kx + B)] = cexp(I * 2.0 * PI * u * (mpz - Dz));   /* (8e) */
            for (int iz = 0; iz < Mz; ++iz)                                     /* (8k) */
                dz[((size_t)iz * W + (ky + B)) * W + (kx + B)] =
                    orc_dirichlet(Mz, (iz + kzlo) / Mzd + u);
        }
    for (int iz = 0; iz < Mz; ++iz)
        for (int jy = 0; jy < W; ++jy)
            for (int jx = 0; jx < W; ++jx) {
                cplx Q = 0.0;                                                   /* (8a) */
                for (int ky = 0; ky < W; ++ky)
                    for (int kx = 0; kx < W; ++kx)
                        Q += bx[kx] * by[ky] * bz[ky * W + kx] * cx[jx] * cy[jy] * cz[iz] *
                             dx[jx * W + kx] * dy[jy * W + ky] *
                             dz[((size_t)iz * W + ky) * W + kx];
                size_t o = ((size_t)iz * W + jy) * W + jx;
                h_re[o] = creal(norm * Q);
                h_im[o] = cimag(norm * Q);
            }
    free(bx); free(by); free(cx); free(cy); free(cz); free(bz); free(dx); free(dy); free(dz);
}

/* ---------------------------------------------------------------------- */
typedef struct {
    int M, K, Mz, kzlo, B, mpx, mpy, mpz, L, nb, nbp;
    double alpha, vmax, vstep;
    int hp_lines;         /* 0: zero bins kx=ky=0; 1: zero every kx=0 or ky=0 bin */
    double *cosR;         /* [L*L][nb]: Re F*(l,k) sqrt(N), Eq. (10), lz = 1 */
    double *hpef_re;      /* [L*L][nbp] PEF coefficients per grid velocity */
    double *hpef_im;
} orc_ctx;

static int wrapk(int k, int lo, int n)
{   /* map integer bin k into [lo, lo+n) modulo n */
    int r = (k - lo) % n;
    if (r < 0) r += n;
    return r + lo;
}

orc_ctx *orc_create(int M, int Mz, int B, int mpz, double alpha, double vmax,
                    double vstep, int hp_lines)
{
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->M = M;
    c->K = (M - 1) / 2;
    c->Mz = Mz;
    c->kzlo = -((Mz - 1) / 2);
    c->B = B;
    c->mpx = c->K;   /* linear-phase spatial delay m'x = Kx, m'y = Ky (Sec. 3) */
    c->mpy = c->K;
    c->mpz = mpz;
    c->alpha = alpha;
    c->vmax = vmax;
    c->vstep = vstep;
    c->L = (int)nearbyint(2.0 * vmax / vstep) + 1;
    c->nb = M * M * Mz;
    c->nbp = (2 * B + 1) * (2 * B + 1) * Mz;
    c->hp_lines = hp_lines;
    int L = c->L, nb = c->nb;
    c->cosR = (double *)malloc(sizeof(double) * (size_t)L * L * nb);
    for (int gy = 0; gy < L; ++gy)
        for (int gx = 0; gx < L; ++gx) {
            double lx = -vmax + gx * vstep, ly = -vmax + gy * vstep, lz = 1.0;
            double *row = c->cosR + ((size_t)gy * L + gx) * nb;
            for (int iz = 0; iz < Mz; ++iz)
                for (int iy = 0; iy < M; ++iy)
                    for (int ix = 0; ix < M; ++ix) {
                        double kx = ix - c->K, ky = iy - c->K, kz = iz + c->kzlo;
                        double ph = 2.0 * PI * (kx * lx / M + ky * ly / M + kz * lz / Mz);
                        row[((size_t)iz * M + iy) * M + ix] = creal(cexp(-I * ph));
                    }
        }
    c->hpef_re = (double *)malloc(sizeof(double) * (size_t)L * L * c->nbp);
    c->hpef_im = (double *)malloc(sizeof(double) * (size_t)L * L * c->nbp);
    #pragma omp parallel for schedule(dynamic)
    for (int g = 0; g < L * L; ++g) {
        double vx = -vmax + (g % L) * vstep, vy = -vmax + (g / L) * vstep;
        orc_pef_design(M, Mz, B, c->mpx, c->mpy, mpz, vx, vy,
                       c->hpef_re + (size_t)g * c->nbp, c->hpef_im + (size_t)g * c->nbp);
    }
    return c;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->cosR);
    free(c->hpef_re);
    free(c->hpef_im);
    free(c);
}

int orc_grid_len(const orc_ctx *c) { return c->L; }

/* Hann window as a frequency-domain convolution along one axis (Sec. 2,
 * after Eq. (9)): for w(m) = 1/2 + 1/2 cos(2 pi (m - D)/n), D = (n-1)/2,
 *   S'(k) = 1/2 S(k) + 1/4 exp(-j2pi D/n) S(k+1) + 1/4 exp(+j2pi D/n) S(k-1),
 * bins taken modulo n.  'get' strides through one line of the cube.        */
static void hann_line(cplx *v, int n, int lo, int stride, cplx *tmp)
{
    double D = (n - 1) / 2.0;
    cplx ap = cexp(-I * 2.0 * PI * D / n), am = cexp(I * 2.0 * PI * D / n);
    for (int i = 0; i < n; ++i) tmp[i] = v[(size_t)i * stride];
    for (int i = 0; i < n; ++i) {
        int k = i + lo;
        int ip = wrapk(k + 1, lo, n) - lo, im = wrapk(k - 1, lo, n) - lo;
        v[(size_t)i * stride] = 0.5 * tmp[i] + 0.25 * ap * tmp[ip] + 0.25 * am * tmp[im];
    }
}

/*
 * Run the whole preprocessor over frames[T][H][W] for the output pixels of
 * the crop [y0, y0+h) x [x0, x0+w).  Reads outside the frame clamp to the
 * edge, so a crop gives exactly the full-frame result for its pixels.
 *
 * Per frame t, in the paper's order (Sec. 1-2):
 *   1. spatial SDFT along rows, then along columns (comb + resonator);
 *   2. deadbeat observer per spatial bin over time;   -> S(k; n), Eq. (6)-(7)
 *   3. high-pass: S(0,0,kz) = 0;  Hann convolution in kx, ky, kz;
 *   4. P = conj(S') S', Eq. (9);
 *   5. R(l) = sqrt(N) sum_k F*(l,k) P(k), Eq. (10), on the lz = 1 slice;
 *   6. R' = (1-alpha) R + alpha R'_prev;  argmax -> velocity (lz = 1);
 *   7. Ihat = sum_{|kx|,|ky|<=B, all kz} H(k; m', v) S(k), Eq. (4), with H
 *      from Eq. (8);  E = I(p, t - m'z) - Re(Ihat)   (Eq. (1) context).
 *
 * Outputs (any may be NULL):
 *   whitened [T][h][w]      E for frame t - m'z, stored at index t (NaN for t < m'z)
 *   vel_index [T][h][w]     flat grid index of the argmax of R' at frame t
 *   vel_override [T][h][w]  if given, the PEF uses this grid index instead
 *   fixed_v[2]              if given, the PEF uses this (vx, vy) everywhere
 *   spec_re/im [nspec][h][w][nb]   S(k; n) at frames spec_t[]
 *   pow_out [nspec][h][w][nb]      P(k; n) at frames spec_t[]
 *   specw_re/im [nspec][h][w][nb]  high-passed, Hann-windowed spectrum at spec_t[]
 *   rs_out  [nspec][h][w][L*L]     R'(l; n) at frames spec_t[]
 */
int orc_run(const orc_ctx *c, const float *frames, int T, int H, int W,
            int y0, int x0, int h, int w,
            double *whitened, int *vel_index, const int *vel_override,
            const double *fixed_v,
            const int *spec_t, int nspec, double *spec_re, double *spec_im,
            double *pow_out, double *rs_out, double *specw_re, double *specw_im,
            int nthreads)
{
    const int M = c->M, K = c->K, Mz = c->Mz, kzlo = c->kzlo, L = c->L;
    const int nb = c->nb, nbp = c->nbp, B = c->B, WB = 2 * B + 1;
    const int hx = h + 2 * K, wx = w + 2 * K;   /* extended rows / columns */
    const double N = (double)M * M * Mz;
    if (h <= 0 || w <= 0 || T <= 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    /* persistent state: observer per pixel per spatial bin, smoother per pixel */
    cplx *obs = (cplx *)calloc((size_t)h * w * M * M * Mz, sizeof(cplx));
    double *rsm = (double *)calloc((size_t)h * w * L * L, sizeof(double));
    /* per-frame work buffers */
    cplx *Xr = (cplx *)malloc(sizeof(cplx) * (size_t)hx * M * w); /* [row][kx][px] */
    cplx *Sxy = (cplx *)malloc(sizeof(cplx) * (size_t)h * w * M * M); /* [py][px][ky][kx] */
    double *fixed_re = NULL, *fixed_im = NULL;
    if (fixed_v) {
        fixed_re = (double *)malloc(sizeof(double) * nbp);
        fixed_im = (double *)malloc(sizeof(double) * nbp);
        orc_pef_design(M, Mz, B, c->mpx, c->mpy, c->mpz, fixed_v[0], fixed_v[1],
                       fixed_re, fixed_im);
    }

    for (int t = 0; t < T; ++t) {
        const float *fr = frames + (size_t)t * H * W;
        int spec_slot = -1;
        for (int s = 0; s < nspec; ++s)
            if (spec_t[s] == t) spec_slot = s;

        /* 1a. SDFT along each (clamped) row, for every kx */
        #pragma omp parallel for schedule(static)
        for (int rr = 0; rr < hx; ++rr) {
            int yr = y0 - K + rr;
            yr = yr < 0 ? 0 : (yr >= H ? H - 1 : yr);
            cplx *e = (cplx *)malloc(sizeof(cplx) * wx);
            cplx *o = (cplx *)malloc(sizeof(cplx) * wx);
            for (int nn = 0; nn < wx; ++nn) {
                int xs = x0 - K + nn;
                xs = xs < 0 ? 0 : (xs >= W ? W - 1 : xs);
                e[nn] = (double)fr[(size_t)yr * W + xs];
            }
            for (int ix = 0; ix < M; ++ix) {
                orc_sdft_line(e, wx, M, ix - K, o);
                for (int px = 0; px < w; ++px)   /* window origin at nn = px + 2K */
                    Xr[((size_t)rr * M + ix) * w + px] = o[px + 2 * K];
            }
            free(e);
            free(o);
        }
        /* 1b. SDFT along each column of every kx plane, for every ky */
        #pragma omp parallel for schedule(static)
        for (int px = 0; px < w; ++px) {
            cplx *e = (cplx *)malloc(sizeof(cplx) * hx);
            cplx *o = (cplx *)malloc(sizeof(cplx) * hx);
            for (int ix = 0; ix < M; ++ix) {
                for (int rr = 0; rr < hx; ++rr) e[rr] = Xr[((size_t)rr * M + ix) * w + px];
                for (int iy = 0; iy < M; ++iy) {
                    orc_sdft_line(e, hx, M, iy - K, o);
                    for (int py = 0; py < h; ++py)
                        Sxy[(((size_t)py * w + px) * M + iy) * M + ix] = o[py + 2 * K];
                }
            }
            free(e);
            free(o);
        }

        /* 2-7 per pixel */
        #pragma omp parallel for schedule(static)
        for (int py = 0; py < h; ++py) {
            cplx *S = (cplx *)malloc(sizeof(cplx) * nb);
            cplx *Sp = (cplx *)malloc(sizeof(cplx) * nb);
            cplx *a = (cplx *)malloc(sizeof(cplx) * Mz);
            cplx *tmp = (cplx *)malloc(sizeof(cplx) * (M > Mz ? M : Mz));
            double *P = (double *)malloc(sizeof(double) * nb);
            double *R = (double *)malloc(sizeof(double) * L * L);
            for (int px = 0; px < w; ++px) {
                size_t pix = (size_t)py * w + px;
                /* 2. deadbeat observer per spatial bin -> S(k; n) */
                for (int iy = 0; iy < M; ++iy)
                    for (int ix = 0; ix < M; ++ix) {
                        cplx *s = obs + (pix * M * M + (size_t)iy * M + ix) * Mz;
                        orc_observer_step(s, Mz, kzlo, Sxy[(pix * M + iy) * M + ix], a);
                        for (int iz = 0; iz < Mz; ++iz)  /* S = (1/sqrt N) Mz a */
                            S[((size_t)iz * M + iy) * M + ix] = a[iz] * ((double)Mz / sqrt(N));
                    }
                /* 3. high-pass then Hann convolution along kx, ky, kz */
                memcpy(Sp, S, sizeof(cplx) * nb);
                for (int iz = 0; iz < Mz; ++iz)
                    for (int iy = 0; iy < M; ++iy)
                        for (int ix = 0; ix < M; ++ix) {
                            int zero = (ix == K && iy == K);
                            if (c->hp_lines) zero = (ix == K || iy == K);
                            if (zero) Sp[((size_t)iz * M + iy) * M + ix] = 0.0;
                        }
                for (int iz = 0; iz < Mz; ++iz)
                    for (int iy = 0; iy < M; ++iy)
                        hann_line(Sp + ((size_t)iz * M + iy) * M, M, -K, 1, tmp);
                for (int iz = 0; iz < Mz; ++iz)
                    for (int ix = 0; ix < M; ++ix)
                        hann_line(Sp + (size_t)iz * M * M + ix, M, -K, M, tmp);
                for (int iy = 0; iy < M; ++iy)
                    for (int ix = 0; ix < M; ++ix)
                        hann_line(Sp + (size_t)iy * M + ix, Mz, kzlo, M * M, tmp);
                /* 4. power, Eq. (9) */
                for (int b = 0; b < nb; ++b) P[b] = creal(conj(Sp[b]) * Sp[b]);
                /* 5. autocorrelation on the lz = 1 slice, Eq. (10) (real part) */
                for (int g = 0; g < L * L; ++g) {
                    const double *cr = c->cosR + (size_t)g * nb;
                    double acc = 0.0;
                    for (int b = 0; b < nb; ++b) acc += cr[b] * P[b];
                    R[g] = acc;
                }
                /* 6. first-order smoothing and argmax (ties -> lowest index) */
                double *rs = rsm + pix * L * L;
                int best = 0;
                for (int g = 0; g < L * L; ++g) {
                    rs[g] = (1.0 - c->alpha) * R[g] + c->alpha * rs[g];
                    if (rs[g] > rs[best]) best = g;
                }
                size_t tp = (size_t)t * h * w + pix;
                if (vel_index) vel_index[tp] = best;
                /* 7. velocity-tuned PEF in the frequency domain, Eq. (4) */
                int g = vel_override ? vel_override[tp] : best;
                const double *hr = fixed_v ? fixed_re : c->hpef_re + (size_t)g * nbp;
                const double *hi = fixed_v ? fixed_im : c->hpef_im + (size_t)g * nbp;
                cplx Ihat = 0.0;
                for (int iz = 0; iz < Mz; ++iz)
                    for (int jy = 0; jy < WB; ++jy)
                        for (int jx = 0; jx < WB; ++jx) {
                            size_t o = ((size_t)iz * WB + jy) * WB + jx;
                            cplx Hk = hr[o] + I * hi[o];
                            Ihat += Hk * S[((size_t)iz * M + (jy - B + K)) * M + (jx - B + K)];
                        }
                if (whitened) {
                    int td = t - c->mpz;
                    if (td >= 0) {
                        double Iin = frames[(size_t)td * H * W + (size_t)(y0 + py) * W + (x0 + px)];
                        whitened[tp] = Iin - creal(Ihat);
                    } else {
                        whitened[tp] = NAN;
                    }
                }
                if (spec_slot >= 0) {
                    size_t so = ((size_t)spec_slot * h * w + pix) * nb;
                    for (int b = 0; b < nb; ++b) {
                        if (spec_re) spec_re[so + b] = creal(S[b]);
                        if (spec_im) spec_im[so + b] = cimag(S[b]);
                        if (pow_out) pow_out[so + b] = P[b];
                        if (specw_re) specw_re[so + b] = creal(Sp[b]);
                        if (specw_im) specw_im[so + b] = cimag(Sp[b]);
                    }
                    if (rs_out)
                        memcpy(rs_out + ((size_t)spec_slot * h * w + pix) * L * L, rs,
                               sizeof(double) * L * L);
                }
            }
            free(S); free(Sp); free(a); free(tmp); free(P); free(R);
        }
    }
    free(obs); free(rsm); free(Xr); free(Sxy);
    free(fixed_re); free(fixed_im);
    return 0;
}
