/*
 * reed_oracle.c -- plain, slow FP64 CPU reference of the REED-MD track step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no source with the CUDA path:
 * every constant, table and formula below is written out here on its own.
 *
 * What it computes (Jeon & Gronbech-Jensen, Sec. 2, "Review of the REED-MD
 * Algorithm"):
 *   - ion-target forces from the universal ZBL screened Coulomb potential
 *     (Sec. 2, "First"), truncated with a C2 quintic taper;
 *   - a domain-following window of n^3 unit cells around the ion; when the
 *     ion leaves its cell the window moves, cells behind are dropped and new
 *     statistically-realised cells are created ahead (Sec. 2, "Second";
 *     Fig. "moving cell"), thermal disorder as Gaussian site displacements
 *     (Sec. 4.1);
 *   - electronic stopping as a velocity-proportional drag on the ion
 *     (Sec. 2, "Third"; Lindhard-Scharff magnitude, optional local-density
 *     factor);
 *   - a velocity Verlet integrator with adaptive time step (Sec. 2, Fig.
 *     "dt_E"; time unit 10.18 fs);
 *   - rare-event enhancement: a track that first passes a cloning depth is
 *     split in two, each copy carrying half the weight (Sec. 2, Fig. "split");
 *     cloning depths are frozen during a track (Sec. 3);
 *   - the weighted range (stopping depth) histogram (Sec. 2);
 *   - the paper's own runs (Sec. 4.1, 4.2): recoils starting on a lattice
 *     site of a bulk crystal in a random direction, their range measured
 *     from the start.
 * Target-target forces (Sec. 1: "all the relevant atomic interactions are
 * included every time step") are Tersoff Si(C) [PRB 38, 9902 (1988)] with a
 * ZBL blend at short range, or Buckingham pair terms splined to ZBL.
 *
 * Where the paper defers to its references, the readings taken are listed in
 * the project's design notes; each is marked "reading:" below.
 *
 * Parity unpinned: the O-O Buckingham values, which no test property is
 * sensitive to (the Ce-O values are pinned by the CeO2 lattice constant they
 * reproduce with formal charges; the Lindhard-Scharff magnitude against the
 * LSS reduced-unit form).
 *
 * Units: Angstrom, eV, amu; time unit tau = sqrt(amu A^2 / eV) = 10.1805 fs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_E2 14.399645          /* e^2/(4 pi eps0), eV*A */
#define O_BOHR 0.529177         /* Bohr radius, A */
#define O_TAU_FS 10.180505710   /* sqrt(amu*A^2/eV) in fs */
#define O_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Parameters (the oracle's own layout; mirrored by oracle/oracle.py)       */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* ion */
    double Z1, M1;
    /* target lattice: 0 diamond, 1 fluorite, -1 explicit atoms (no lattice) */
    int lattice;
    int n;            /* cells per window edge */
    int margin;       /* frozen outer cell layers (0 or 1) */
    int nspec;
    /* target geometry: 0 = surface (target z >= 0, (001) surface), 1 = bulk
     * (infinite crystal; the recoil's own site, basis atom 0 of cell
     * (0,0,0), is vacant) */
    int target;
    double a;         /* lattice constant, A */
    double sigma;     /* thermal displacement per Cartesian coordinate, A */
    double Z2[2], M2[2];
    /* ion-target potential */
    double rc, rt;    /* cutoff and taper start */
    int screening;    /* 1 = ZBL universal screening, 0 = bare Coulomb */
    int tt;           /* target-target: 0 none, 1 Tersoff, 2 Buckingham */
    double spline_c[6];  /* ZBL correction coefficients (0 = pure ZBL) */
    /* Tersoff: A B lam1 lam2 beta n c d h R D */
    double ters[11];
    double blend_lo, blend_hi;   /* Tersoff->ZBL blend window */
    /* Buckingham per species pair (00, 01, 11): A, rho, C */
    double bk_A[3], bk_rho[3], bk_C[3];
    double bk_rc, bk_rt, bk_lo, bk_hi;  /* cutoff, taper start, ZBL blend */
    /* electronic stopping */
    double s_e, s_loc, lam_loc;
    /* integrator */
    double dt_max;    /* tau */
    double dx_max;    /* A */
    double e_stop;    /* eV */
    int64_t step_cap;
    /* beam */
    double E0, tilt, rot_lo, rot_hi;  /* eV, degrees */
    int beam_mode;    /* 0: fixed tilt, rotation U[lo,hi); 1: cone of half-angle tilt;
                         2: recoil from the origin site, direction uniform on the sphere */
    /* cloning depths and histogram */
    int nthr;
    double thr[16];
    int nbins;
    double bin_w;
    /* cumulative damage map (reading): dn^3 voxels of dvox A, origin
     * (-dn dvox / 2, -dn dvox / 2, 0) -- in a bulk target (-dn dvox / 2) on
     * all three axes; atoms with KE > dmin deposit w KE */
    int dn;
    double dvox, dmin;
    /* energy term of the adaptive step (eV per step; 0 = off) */
    double de_max;
    /* damage feedback (reading, see o_cell_atoms): on when fb_ec > 0 and
     * fb_map is set; fb_map holds the dn^3 (+ overflow) map as it stood when
     * the run started */
    double dose_scale, fb_ec, sigma_am;
    const double* fb_map;
    /* the energy term never shortens the fastest particle's step below dx_min
     * (A; reading, see o_pick_dt) */
    double dx_min;
} o_params;

typedef struct {
    uint64_t id, primary;
    double z, t;
    int64_t steps;
    int32_t level, status;
} o_record;

enum { O_ALIVE = 0, O_STOPPED = 1, O_BACK = 2, O_TRUNC = 3 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the      */
/* published definition: 10 rounds of two 32x32->64 multiplies with a Weyl  */
/* key schedule.                                                            */
/* ------------------------------------------------------------------------ */
void o_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* SplitMix64 output mixer (Steele, Lea, Flood, OOPSLA'14). */
static uint64_t o_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* reading: per-track Philox key = mix64(seed + golden*(id+1)). */
uint64_t o_track_key(uint64_t seed, uint64_t id)
{
    return o_mix64(seed + 0x9E3779B97F4A7C15ull * (id + 1ull));
}

/* reading: the clone spawned at cloning level L gets id mix64(parent ^ ...). */
uint64_t o_child_id(uint64_t parent, int level)
{
    return o_mix64(parent ^ (0xD1B54A32D192ED03ull * (uint64_t)(level + 1)));
}

#define O_TAG_CELL 1u
#define O_TAG_LAUNCH 2u
#define O_TAG_DAMAGE 3u

static void o_draw(uint64_t key, int32_t ix, int32_t iy, int32_t iz, uint32_t word, uint32_t out[4])
{
    uint32_t c[4] = {(uint32_t)ix, (uint32_t)iy, (uint32_t)iz, word};
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
    o_philox(c, k, out);
}

static double o_unit(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Three i.i.d. standard normals from one Philox block (Box-Muller). */
void o_gauss3(const uint32_t w[4], double g[3])
{
    double r1 = sqrt(-2.0 * log(o_unit(w[0])));
    double a1 = 2.0 * O_PI * o_unit(w[1]);
    double r2 = sqrt(-2.0 * log(o_unit(w[2])));
    double a2 = 2.0 * O_PI * o_unit(w[3]);
    g[0] = r1 * cos(a1);
    g[1] = r1 * sin(a1);
    g[2] = r2 * cos(a2);
}

/* ------------------------------------------------------------------------ */
/* Lattices (Sec. 2: 12-atom fluorite cell; diamond cubic for Si)           */
/* ------------------------------------------------------------------------ */
static const double O_DIAMOND[8][3] = {
    {0.00, 0.00, 0.00}, {0.00, 0.50, 0.50}, {0.50, 0.00, 0.50}, {0.50, 0.50, 0.00},
    {0.25, 0.25, 0.25}, {0.25, 0.75, 0.75}, {0.75, 0.25, 0.75}, {0.75, 0.75, 0.25}};
static const double O_FLUORITE[12][3] = {
    {0.00, 0.00, 0.00}, {0.00, 0.50, 0.50}, {0.50, 0.00, 0.50}, {0.50, 0.50, 0.00},
    {0.25, 0.25, 0.25}, {0.75, 0.25, 0.25}, {0.25, 0.75, 0.25}, {0.25, 0.25, 0.75},
    {0.75, 0.75, 0.25}, {0.75, 0.25, 0.75}, {0.25, 0.75, 0.75}, {0.75, 0.75, 0.75}};

int o_basis_count(int lattice) { return lattice == 1 ? 12 : (lattice == 0 ? 8 : 0); }

static int o_basis_species(int lattice, int b) { return (lattice == 1 && b >= 4) ? 1 : 0; }

/* reading (damage feedback; the paper feeds cumulative damage back to the
 * tracks, Sec. 1 and 3, without giving the mechanism): a cell created where
 * the cumulative damage map holds D (eV) in the voxel of the cell's centre
 * is amorphous with probability 1 - exp(-e / fb_ec), e = dose_scale * D / N
 * the energy deposited per target atom (N = atoms of the perfect lattice in
 * one voxel); an amorphous cell's atoms are displaced by sigma_am instead of
 * sigma.  The decision uses its own Philox block (tag 3) of the cell. */
static double o_cell_sigma(const o_params* P, uint64_t key, int32_t ix, int32_t iy, int32_t iz)
{
    if (!(P->fb_ec > 0.0) || !P->fb_map || P->dn <= 0) return P->sigma;
    double half = 0.5 * P->dn * P->dvox;
    double zhalf = P->target == 1 ? half : 0.0;
    int v[3];
    double c[3] = {(ix + 0.5) * P->a + half, (iy + 0.5) * P->a + half, (iz + 0.5) * P->a + zhalf};
    for (int d = 0; d < 3; ++d) {
        v[d] = (int)floor(c[d] / P->dvox);
        if (v[d] < 0 || v[d] >= P->dn) return P->sigma;
    }
    double D = P->fb_map[((size_t)v[0] * P->dn + v[1]) * P->dn + v[2]];
    double cells_per_voxel = pow(P->dvox / P->a, 3.0);
    double N = o_basis_count(P->lattice) * cells_per_voxel;
    double e = P->dose_scale * D / N;
    double pam = 1.0 - exp(-e / P->fb_ec);
    uint32_t w[4];
    o_draw(key, ix, iy, iz, O_TAG_DAMAGE, w);
    return o_unit(w[0]) < pam ? P->sigma_am : P->sigma;
}

/* Atoms of absolute cell (ix,iy,iz), absolute coordinates.  Cells with
 * iz < 0 lie above the surface and are empty (target occupies z >= 0).
 * reading (the paper's UO2 runs start from a lattice site, Sec. 4.1): a bulk
 * target fills space, and the site the recoil starts from -- basis atom 0 of
 * cell (0,0,0) -- is empty in every realisation of that cell.
 * Returns the number of atoms written; bas (may be NULL) receives each
 * atom's basis index. */
static int o_cell_atoms_b(const o_params* P, uint64_t key, int32_t ix, int32_t iy, int32_t iz,
                          double* xyz, int* sp, int* bas)
{
    if (P->target != 1 && iz < 0) return 0;
    int nb = o_basis_count(P->lattice);
    const double(*B)[3] = P->lattice == 1 ? O_FLUORITE : O_DIAMOND;
    double sig = o_cell_sigma(P, key, ix, iy, iz);
    int m = 0;
    for (int b = 0; b < nb; ++b) {
        if (P->target == 1 && b == 0 && ix == 0 && iy == 0 && iz == 0) continue;   /* the recoil's site */
        double g[3] = {0.0, 0.0, 0.0};
        if (sig > 0.0) {
            uint32_t w[4];
            o_draw(key, ix, iy, iz, ((uint32_t)b << 4) | O_TAG_CELL, w);
            o_gauss3(w, g);
        }
        xyz[3 * m + 0] = (ix + B[b][0]) * P->a + sig * g[0];
        xyz[3 * m + 1] = (iy + B[b][1]) * P->a + sig * g[1];
        xyz[3 * m + 2] = (iz + B[b][2]) * P->a + sig * g[2];
        sp[m] = o_basis_species(P->lattice, b);
        if (bas) bas[m] = b;
        ++m;
    }
    return m;
}

int o_cell_atoms(const o_params* P, uint64_t key, int32_t ix, int32_t iy, int32_t iz, double* xyz, int* sp)
{
    return o_cell_atoms_b(P, key, ix, iy, iz, xyz, sp, NULL);
}

/* ------------------------------------------------------------------------ */
/* Potentials                                                               */
/* ------------------------------------------------------------------------ */
/* ZBL universal screening function coefficients (Ziegler, Biersack,
 * Littmark, "The Stopping and Range of Ions in Solids", 1985). */
static const double O_ZC[4] = {0.18175, 0.50986, 0.28022, 0.02817};
static const double O_ZD[4] = {3.19980, 0.94229, 0.40290, 0.20162};

double o_zbl_screen_length(double Z1, double Z2)
{
    return 0.8854 * O_BOHR / (pow(Z1, 0.23) + pow(Z2, 0.23));
}

/* Cubic B-spline basis on the knots of ln r used by the ZBL correction.
 * reading: six uniform cubic B-splines centred on ln r_i for
 * r_i = {0.2,0.35,0.6,1.0,1.7,3.0} A, width set by the mean knot spacing. */
static const double O_KNOTS[6] = {0.2, 0.35, 0.6, 1.0, 1.7, 3.0};

static double o_bspline3(double u, double* du)
{
    /* centred cubic B-spline of unit spacing, support |u| < 2 */
    double au = fabs(u), s = u < 0 ? -1.0 : 1.0;
    if (au >= 2.0) { *du = 0.0; return 0.0; }
    if (au >= 1.0) {
        double q = 2.0 - au;
        *du = -s * 0.5 * q * q;
        return q * q * q / 6.0;
    }
    *du = s * (-2.0 * au + 1.5 * au * au);
    return 2.0 / 3.0 - au * au + 0.5 * au * au * au;
}

/* returns log-correction c(r) = sum_i c_i B_i(ln r) and its r-derivative */
static double o_spline_corr(const double* c, double r, double* dcdr)
{
    double h = (log(O_KNOTS[5]) - log(O_KNOTS[0])) / 5.0;
    double lr = log(r), s = 0.0, ds = 0.0;
    for (int i = 0; i < 6; ++i) {
        if (c[i] == 0.0) continue;
        double du, b = o_bspline3((lr - log(O_KNOTS[i])) / h, &du);
        s += c[i] * b;
        ds += c[i] * du / h;
    }
    *dcdr = ds / r;
    return s;
}

/* Bare ZBL V(r) and dV/dr for charges Z1, Z2; screening optional. */
void o_zbl(double Z1, double Z2, int screening, double r, double* V, double* dV)
{
    double k = Z1 * Z2 * O_E2;
    if (!screening) {
        *V = k / r;
        *dV = -k / (r * r);
        return;
    }
    double au = o_zbl_screen_length(Z1, Z2);
    double x = r / au, phi = 0.0, dphi = 0.0;
    for (int i = 0; i < 4; ++i) {
        double e = exp(-O_ZD[i] * x);
        phi += O_ZC[i] * e;
        dphi -= O_ZC[i] * O_ZD[i] * e;
    }
    *V = k * phi / r;
    *dV = k * (dphi / (au * r) - phi / (r * r));
}

/* C2 quintic taper: 1 below rt, 0 above rc. */
static double o_taper(double r, double rt, double rc, double* dS)
{
    if (r <= rt) { *dS = 0.0; return 1.0; }
    if (r >= rc) { *dS = 0.0; return 0.0; }
    double w = rc - rt, t = (r - rt) / w;
    double t2 = t * t, t3 = t2 * t;
    *dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t2 * t2) / w;
    return 1.0 - 10.0 * t3 + 15.0 * t2 * t2 - 6.0 * t3 * t2;
}

/* Ion-target pair: U = V_ZBL(r) * exp(c(r)) * S(r). */
static double o_ion_pair(const o_params* P, double Z2, double r, double* dU)
{
    double V, dV;
    o_zbl(P->Z1, Z2, P->screening, r, &V, &dV);
    double dc, c = o_spline_corr(P->spline_c, r, &dc);
    double ec = exp(c);
    double dS, S = o_taper(r, P->rt, P->rc, &dS);
    *dU = (dV * ec + V * ec * dc) * S + V * ec * dS;
    return V * ec * S;
}

/* quintic smoothstep that is 1 below lo and 0 above hi (blend weight of ZBL) */
static double o_blend(double r, double lo, double hi, double* ds)
{
    double dS, S = o_taper(r, lo, hi, &dS);
    *ds = dS;
    return S;
}

/* ------------------------------------------------------------------------ */
/* Electronic stopping (Sec. 2 "Third").                                    */
/* reading: F_e = -gamma * (1 + s_loc (rho/rho0 - 1)) * v inside z >= 0;     */
/* gamma = s_e * sum_s N_s k_LS(Z1,Z2_s) sqrt(M1/2), Lindhard-Scharff        */
/* k_LS = 1.212 Z1^(7/6) Z2 / ((Z1^(2/3)+Z2^(2/3))^(3/2) sqrt(M1)).          */
/* ------------------------------------------------------------------------ */
static int o_species_count(int lattice, int s)
{
    if (lattice == 0) return s == 0 ? 8 : 0;
    if (lattice == 1) return s == 0 ? 4 : 8;
    return 0;
}

double o_gamma_ls(const o_params* P)
{
    double g = 0.0;
    if (P->lattice < 0) return 0.0;
    double vol = P->a * P->a * P->a;
    for (int s = 0; s < P->nspec; ++s) {
        double N = o_species_count(P->lattice, s) / vol;
        double Z2 = P->Z2[s];
        double den = pow(pow(P->Z1, 2.0 / 3.0) + pow(Z2, 2.0 / 3.0), 1.5);
        double k = 1.212 * pow(P->Z1, 7.0 / 6.0) * Z2 / (den * sqrt(P->M1));
        g += N * k;
    }
    return P->s_e * g * sqrt(P->M1 / 2.0);
}

double o_rho0(const o_params* P)
{
    if (P->lattice < 0) return 1.0;
    double N = o_basis_count(P->lattice) / (P->a * P->a * P->a);
    return N * 8.0 * O_PI * P->lam_loc * P->lam_loc * P->lam_loc;
}

/* Tallies of finished tracks (per worker thread). */
typedef struct {
    double* hist;      /* nbins + 3: under, over, back -- appended */
    double* damage;    /* dn^3 + 1 (overflow) or NULL */
    double w_trunc;
    double e_dep_sub;  /* weighted KE of dropped atoms below the damage threshold */
    int64_t steps, tracks, clones, shifts;
} o_tally;

/* Deposit the kinetic energy of window atom j (weight w) into the damage map. */
static void o_deposit(const o_params* P, o_tally* T, const double* x, const double* v, double m, double w)
{
    if (!T || !T->damage || P->dn <= 0) return;
    double ke = 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(ke > P->dmin)) {
        T->e_dep_sub += w * ke;
        return;
    }
    double half = 0.5 * P->dn * P->dvox;
    double zhalf = P->target == 1 ? half : 0.0;
    int ix = (int)floor((x[0] + half) / P->dvox);
    int iy = (int)floor((x[1] + half) / P->dvox);
    int iz = (int)floor((x[2] + zhalf) / P->dvox);
    size_t n = (size_t)P->dn;
    if (ix < 0 || iy < 0 || iz < 0 || ix >= P->dn || iy >= P->dn || iz >= P->dn)
        T->damage[n * n * n] += w * ke;
    else
        T->damage[((size_t)ix * n + iy) * n + iz] += w * ke;
}

/* ------------------------------------------------------------------------ */
/* Window / ion state                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int cap, n;
    double* x;   /* 3n */
    double* v;   /* 3n */
    double* f;   /* 3n */
    int* sp;
    int* cell;   /* 3n absolute cell index of the atom's home cell */
    int* bas;    /* basis index */
    int* act;    /* integrated (1) or frozen (0) */
    int A[3];    /* anchor cell index */
} o_win;

typedef struct {
    double x[3], v[3], f[3];
    double rho;      /* local density at x */
    double t;
    double e_elec;   /* energy removed by electronic stopping */
    int level;
    int64_t steps;
    uint64_t id, primary, key;
} o_ion;

static void o_win_alloc(o_win* W, int cap)
{
    memset(W, 0, sizeof(*W));
    W->cap = cap;
    W->x = (double*)calloc(3 * (size_t)cap, sizeof(double));
    W->v = (double*)calloc(3 * (size_t)cap, sizeof(double));
    W->f = (double*)calloc(3 * (size_t)cap, sizeof(double));
    W->sp = (int*)calloc((size_t)cap, sizeof(int));
    W->cell = (int*)calloc(3 * (size_t)cap, sizeof(int));
    W->bas = (int*)calloc((size_t)cap, sizeof(int));
    W->act = (int*)calloc((size_t)cap, sizeof(int));
}

static void o_win_free(o_win* W)
{
    free(W->x); free(W->v); free(W->f); free(W->sp); free(W->cell); free(W->bas); free(W->act);
    memset(W, 0, sizeof(*W));
}

static void o_win_copy(o_win* D, const o_win* S)
{
    D->n = S->n;
    memcpy(D->A, S->A, sizeof(S->A));
    memcpy(D->x, S->x, 3 * sizeof(double) * (size_t)S->n);
    memcpy(D->v, S->v, 3 * sizeof(double) * (size_t)S->n);
    memcpy(D->f, S->f, 3 * sizeof(double) * (size_t)S->n);
    memcpy(D->sp, S->sp, sizeof(int) * (size_t)S->n);
    memcpy(D->cell, S->cell, 3 * sizeof(int) * (size_t)S->n);
    memcpy(D->bas, S->bas, sizeof(int) * (size_t)S->n);
    memcpy(D->act, S->act, sizeof(int) * (size_t)S->n);
}

/* reading (window rule, Fig. "moving cell"): the anchor is the cell that
 * holds the ion (odd n) or the nearest cell corner (even n); the window is
 * cells anchor - n/2 ... anchor - n/2 + n - 1 on each axis. */
static int o_anchor1(const o_params* P, double x)
{
    double h = (P->n % 2 == 0) ? 0.5 : 0.0;
    return (int)floor(x / P->a + h);
}

static int o_lo(const o_params* P, int A) { return A - P->n / 2; }

static int o_cell_active(const o_params* P, const int A[3], const int c[3])
{
    for (int d = 0; d < 3; ++d) {
        int off = c[d] - o_lo(P, A[d]);
        if (off < P->margin || off > P->n - 1 - P->margin) return 0;
    }
    return 1;
}

static int o_in_window(const o_params* P, const int A[3], const int c[3])
{
    for (int d = 0; d < 3; ++d) {
        int off = c[d] - o_lo(P, A[d]);
        if (off < 0 || off > P->n - 1) return 0;
    }
    return 1;
}

static void o_add_cell(const o_params* P, o_win* W, uint64_t key, const int c[3])
{
    double xyz[36];
    int sp[12], bas[12];
    int m = o_cell_atoms_b(P, key, c[0], c[1], c[2], xyz, sp, bas);
    for (int b = 0; b < m; ++b) {
        int j = W->n++;
        for (int d = 0; d < 3; ++d) {
            W->x[3 * j + d] = xyz[3 * b + d];
            W->v[3 * j + d] = 0.0;
            W->f[3 * j + d] = 0.0;
            W->cell[3 * j + d] = c[d];
        }
        W->sp[j] = sp[b];
        W->bas[j] = bas[b];
        W->act[j] = 1;
    }
}

/* Re-anchor the window on the ion: drop atoms whose home cell left the
 * window, create the cells that entered it.  Returns the number of moves. */
static int o_window_update(const o_params* P, o_win* W, const o_ion* I, uint64_t key, o_tally* T)
{
    int A[3];
    for (int d = 0; d < 3; ++d) A[d] = o_anchor1(P, I->x[d]);
    int moved = (A[0] != W->A[0]) || (A[1] != W->A[1]) || (A[2] != W->A[2]);
    if (moved) {
        int old[3] = {W->A[0], W->A[1], W->A[2]};
        /* drop */
        int k = 0;
        for (int j = 0; j < W->n; ++j) {
            if (!o_in_window(P, A, &W->cell[3 * j])) {
                o_deposit(P, T, &W->x[3 * j], &W->v[3 * j], P->M2[W->sp[j]], ldexp(1.0, -I->level));
                continue;
            }
            if (k != j) {
                for (int d = 0; d < 3; ++d) {
                    W->x[3 * k + d] = W->x[3 * j + d];
                    W->v[3 * k + d] = W->v[3 * j + d];
                    W->f[3 * k + d] = W->f[3 * j + d];
                    W->cell[3 * k + d] = W->cell[3 * j + d];
                }
                W->sp[k] = W->sp[j];
                W->bas[k] = W->bas[j];
            }
            ++k;
        }
        W->n = k;
        /* create */
        for (int i = 0; i < P->n; ++i)
            for (int j = 0; j < P->n; ++j)
                for (int l = 0; l < P->n; ++l) {
                    int c[3] = {o_lo(P, A[0]) + i, o_lo(P, A[1]) + j, o_lo(P, A[2]) + l};
                    if (!o_in_window(P, old, c)) o_add_cell(P, W, key, c);
                }
        W->A[0] = A[0]; W->A[1] = A[1]; W->A[2] = A[2];
    }
    for (int j = 0; j < W->n; ++j) W->act[j] = o_cell_active(P, W->A, &W->cell[3 * j]);
    return moved;
}

static void o_window_init(const o_params* P, o_win* W, const o_ion* I, uint64_t key)
{
    W->n = 0;
    for (int d = 0; d < 3; ++d) W->A[d] = o_anchor1(P, I->x[d]);
    for (int i = 0; i < P->n; ++i)
        for (int j = 0; j < P->n; ++j)
            for (int l = 0; l < P->n; ++l) {
                int c[3] = {o_lo(P, W->A[0]) + i, o_lo(P, W->A[1]) + j, o_lo(P, W->A[2]) + l};
                o_add_cell(P, W, key, c);
            }
    for (int j = 0; j < W->n; ++j) W->act[j] = o_cell_active(P, W->A, &W->cell[3 * j]);
}

/* ------------------------------------------------------------------------ */
/* Forces                                                                   */
/* ------------------------------------------------------------------------ */
static double o_dist(const double* a, const double* b, double r[3])
{
    r[0] = b[0] - a[0]; r[1] = b[1] - a[1]; r[2] = b[2] - a[2];
    return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
}

/* Tersoff cutoff function fc and derivative. */
static double o_fc(double r, double R, double D, double* dfc)
{
    if (r < R - D) { *dfc = 0.0; return 1.0; }
    if (r > R + D) { *dfc = 0.0; return 0.0; }
    double q = 0.5 * O_PI * (r - R) / D;
    *dfc = -0.25 * O_PI / D * cos(q);
    return 0.5 - 0.5 * sin(q);
}

static double o_g(double c, double C, double Dd, double H, double* dg)
{
    double q = H - c, den = Dd * Dd + q * q;
    *dg = -2.0 * C * C * q / (den * den);
    return 1.0 + C * C / (Dd * Dd) - C * C / den;
}

/* Tersoff energy with ZBL blend; scatter forces into f (3n). All n atoms
 * are included in the energy.  The partners of atom i are the atoms j != i
 * with r_ij < R + D, found by brute force over all n atoms and kept in
 * ascending index order; the sums over j and over the third atom k run over
 * that list, which visits exactly the terms (and in the same order) of a
 * loop over all atoms that skips those beyond the cutoff. */
static double o_tersoff(const o_params* P, int n, const double* x, double* f)
{
    const double *T = P->ters;
    const double A = T[0], Bt = T[1], l1 = T[2], l2 = T[3], beta = T[4], nn = T[5];
    const double C = T[6], Dd = T[7], H = T[8], R = T[9], D = T[10];
    const double rcut = R + D;
    double E = 0.0;
    double Zs = P->Z2[0];
    double bn = pow(beta, nn);
    int* cnt = (int*)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    int* nbr = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double rv[3];
            if (o_dist(&x[3 * i], &x[3 * j], rv) < rcut) nbr[(size_t)i * n + cnt[i]++] = j;
        }
    for (int i = 0; i < n; ++i) {
        const int* Ni = nbr + (size_t)i * n;
        for (int jj = 0; jj < cnt[i]; ++jj) {
            const int j = Ni[jj];
            double rij_v[3], rij = o_dist(&x[3 * i], &x[3 * j], rij_v);
            /* zeta_ij */
            double zeta = 0.0;
            for (int kk = 0; kk < cnt[i]; ++kk) {
                const int k = Ni[kk];
                if (k == j) continue;
                double rik_v[3], rik = o_dist(&x[3 * i], &x[3 * k], rik_v);
                double dfc, fck = o_fc(rik, R, D, &dfc);
                double cs = (rij_v[0] * rik_v[0] + rij_v[1] * rik_v[1] + rij_v[2] * rik_v[2]) / (rij * rik);
                double dg;
                zeta += fck * o_g(cs, C, Dd, H, &dg);
            }
            double bz = 1.0 + bn * pow(zeta, nn);
            double b = pow(bz, -0.5 / nn);
            double dbdz = (zeta > 0.0) ? -0.5 * bn * pow(zeta, nn - 1.0) * pow(bz, -0.5 / nn - 1.0) : 0.0;
            double dfc, fc = o_fc(rij, R, D, &dfc);
            double fR = A * exp(-l1 * rij), dfR = -l1 * fR;
            double fA = -Bt * exp(-l2 * rij), dfA = -l2 * fA;
            double VT = fc * (fR + b * fA);
            double dVT = dfc * (fR + b * fA) + fc * (dfR + b * dfA);
            double Vz, dVz;
            o_zbl(Zs, Zs, 1, rij, &Vz, &dVz);
            double ds, s = o_blend(rij, P->blend_lo, P->blend_hi, &ds);
            double Vij = (1.0 - s) * VT + s * Vz;
            double dV = (1.0 - s) * dVT - ds * VT + ds * Vz + s * dVz;
            E += 0.5 * Vij;
            /* radial part: -dE/dx_j = -0.5 dV rhat_ij */
            for (int d = 0; d < 3; ++d) {
                double u = rij_v[d] / rij;
                f[3 * j + d] -= 0.5 * dV * u;
                f[3 * i + d] += 0.5 * dV * u;
            }
            /* bond-order part: prefactor 0.5 * dV/db * db/dzeta */
            double pre = 0.5 * (1.0 - s) * fc * fA * dbdz;
            if (pre == 0.0) continue;
            for (int kk = 0; kk < cnt[i]; ++kk) {
                const int k = Ni[kk];
                if (k == j) continue;
                double rik_v[3], rik = o_dist(&x[3 * i], &x[3 * k], rik_v);
                double dfck, fck = o_fc(rik, R, D, &dfck);
                double cs = (rij_v[0] * rik_v[0] + rij_v[1] * rik_v[1] + rij_v[2] * rik_v[2]) / (rij * rik);
                double dg, g = o_g(cs, C, Dd, H, &dg);
                for (int d = 0; d < 3; ++d) {
                    double uj = rij_v[d] / rij, uk = rik_v[d] / rik;
                    double dcj = (uk - cs * uj) / rij;   /* d cos / d x_j */
                    double dck = (uj - cs * uk) / rik;   /* d cos / d x_k */
                    double gj = fck * dg * dcj;
                    double gk = dfck * uk * g + fck * dg * dck;
                    f[3 * j + d] -= pre * gj;
                    f[3 * k + d] -= pre * gk;
                    f[3 * i + d] += pre * (gj + gk);
                }
            }
        }
    }
    free(nbr);
    free(cnt);
    return E;
}

/* Buckingham pair energy for species pair index p, with ZBL blend below
 * bk_hi and taper to zero at bk_rc. */
static double o_buck_pair(const o_params* P, int si, int sj, double r, double* dU)
{
    int p = si + sj;   /* 0: 0-0, 1: 0-1, 2: 1-1 */
    double Ab = P->bk_A[p], rho = P->bk_rho[p], Cb = P->bk_C[p];
    double Vb = 0.0, dVb = 0.0;
    if (Ab != 0.0 || Cb != 0.0) {
        double e = Ab * exp(-r / rho);
        double r6 = r * r * r * r * r * r;
        Vb = e - Cb / r6;
        dVb = -e / rho + 6.0 * Cb / (r6 * r);
    }
    double Vz, dVz;
    o_zbl(P->Z2[si], P->Z2[sj], 1, r, &Vz, &dVz);
    double ds, s = o_blend(r, P->bk_lo, P->bk_hi, &ds);
    double V = (1.0 - s) * Vb + s * Vz;
    double dV = (1.0 - s) * dVb - ds * Vb + ds * Vz + s * dVz;
    double dS, S = o_taper(r, P->bk_rt, P->bk_rc, &dS);
    *dU = dV * S + V * dS;
    return V * S;
}

static double o_buckingham(const o_params* P, int n, const double* x, const int* sp, double* f)
{
    double E = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double rv[3], r = o_dist(&x[3 * i], &x[3 * j], rv);
            if (r >= P->bk_rc) continue;
            double dU, U = o_buck_pair(P, sp[i], sp[j], r, &dU);
            E += U;
            for (int d = 0; d < 3; ++d) {
                double u = rv[d] / r;
                f[3 * j + d] -= dU * u;
                f[3 * i + d] += dU * u;
            }
        }
    return E;
}

/* All conservative forces for an ion at xi and n atoms.  f_ion, f (3n) are
 * overwritten.  Returns the potential energy; *rho gets the local density. */
double o_forces(const o_params* P, const double* xi, int with_ion, int n, const double* x,
                const int* sp, double* f_ion, double* f, double* rho)
{
    double E = 0.0, rh = 0.0;
    for (int d = 0; d < 3; ++d) f_ion[d] = 0.0;
    for (int j = 0; j < 3 * n; ++j) f[j] = 0.0;
    if (with_ion) {
        for (int j = 0; j < n; ++j) {
            double rv[3], r = o_dist(xi, &x[3 * j], rv);
            if (r >= P->rc) continue;
            double dU, U = o_ion_pair(P, P->Z2[sp[j]], r, &dU);
            E += U;
            for (int d = 0; d < 3; ++d) {
                double u = rv[d] / r;
                f[3 * j + d] -= dU * u;
                f_ion[d] += dU * u;
            }
            double dS, S = o_taper(r, P->rt, P->rc, &dS);
            rh += S * exp(-r / P->lam_loc);
        }
    }
    if (P->tt == 1) E += o_tersoff(P, n, x, f);
    else if (P->tt == 2) E += o_buckingham(P, n, x, sp, f);
    if (rho) *rho = rh;
    return E;
}

/* ------------------------------------------------------------------------ */
/* Integrator (Sec. 2: Verlet with adaptive time step).                     */
/* reading: dt = min(dt_max, dx_max / v_max), v_max over the ion and the     */
/* integrated atoms; kick-drift-kick with the drag evaluated at the velocity */
/* available at each half kick.  Optional energy term (the paper's step in  */
/* terms of kinetic and collisional energy, reading): dt <= de_max / P, P   */
/* the largest |F . v| (conservative force, velocity) over the ion and the  */
/* integrated atoms at the start of the step.  It never shortens the       */
/* fastest particle's step below dx_min: a step that moves nothing by more   */
/* than a few ulp of a single-precision coordinate would stall an FP32       */
/* window, and the 0.05 A rule already bounds the step from above.           */
/* ------------------------------------------------------------------------ */
static void o_drag(const o_params* P, double gam, double rho0, const o_ion* I, const double* v,
                   const double* x, double rho, double F[3])
{
    double fl = 1.0 + P->s_loc * (rho / rho0 - 1.0);
    double g = (P->target == 1 || x[2] >= 0.0) ? gam * fl : 0.0;   /* inside the target */
    for (int d = 0; d < 3; ++d) F[d] = -g * v[d];
    (void)I;
}

typedef struct {
    double gam, rho0;
} o_consts;

static double o_pick_dt(const o_params* P, const o_ion* I, const o_win* W)
{
    double v2 = I->v[0] * I->v[0] + I->v[1] * I->v[1] + I->v[2] * I->v[2];
    for (int j = 0; j < W->n; ++j) {
        if (!W->act[j]) continue;
        double w2 = W->v[3 * j] * W->v[3 * j] + W->v[3 * j + 1] * W->v[3 * j + 1] +
                    W->v[3 * j + 2] * W->v[3 * j + 2];
        if (w2 > v2) v2 = w2;
    }
    double vmax = sqrt(v2);
    double dt = P->dt_max;
    if (vmax * dt > P->dx_max) dt = P->dx_max / vmax;
    if (P->de_max > 0.0) {
        double pw = fabs(I->f[0] * I->v[0] + I->f[1] * I->v[1] + I->f[2] * I->v[2]);
        for (int j = 0; j < W->n; ++j) {
            if (!W->act[j]) continue;
            double q = fabs(W->f[3 * j] * W->v[3 * j] + W->f[3 * j + 1] * W->v[3 * j + 1] +
                            W->f[3 * j + 2] * W->v[3 * j + 2]);
            if (q > pw) pw = q;
        }
        if (pw * dt > P->de_max) {
            dt = P->de_max / pw;
            if (vmax * dt < P->dx_min) dt = P->dx_min / vmax;
        }
    }
    return dt;
}

static double o_mass(const o_params* P, int s) { return P->M2[s]; }

/* One step.  key: Philox key for newly created cells (<0 lattice: none). */
static double o_step(const o_params* P, const o_consts* K, o_ion* I, o_win* W, uint64_t key,
                     double dt_fixed, int windowing, int* moved, o_tally* T)
{
    double dt = dt_fixed > 0.0 ? dt_fixed : o_pick_dt(P, I, W);
    double Fe[3];
    /* first half kick */
    o_drag(P, K->gam, K->rho0, I, I->v, I->x, I->rho, Fe);
    for (int d = 0; d < 3; ++d) {
        I->v[d] += 0.5 * dt / P->M1 * (I->f[d] + Fe[d]);
        I->e_elec -= 0.5 * dt * Fe[d] * I->v[d];
    }
    for (int j = 0; j < W->n; ++j) {
        if (!W->act[j]) continue;
        double m = o_mass(P, W->sp[j]);
        for (int d = 0; d < 3; ++d) W->v[3 * j + d] += 0.5 * dt / m * W->f[3 * j + d];
    }
    /* drift */
    for (int d = 0; d < 3; ++d) I->x[d] += dt * I->v[d];
    for (int j = 0; j < W->n; ++j) {
        if (!W->act[j]) continue;
        for (int d = 0; d < 3; ++d) W->x[3 * j + d] += dt * W->v[3 * j + d];
    }
    /* window */
    *moved = (windowing && P->lattice >= 0) ? o_window_update(P, W, I, key, T) : 0;
    /* forces at the new positions */
    double U = o_forces(P, I->x, 1, W->n, W->x, W->sp, I->f, W->f, &I->rho);
    /* second half kick */
    o_drag(P, K->gam, K->rho0, I, I->v, I->x, I->rho, Fe);
    for (int d = 0; d < 3; ++d) {
        I->e_elec -= 0.5 * dt * Fe[d] * I->v[d];
        I->v[d] += 0.5 * dt / P->M1 * (I->f[d] + Fe[d]);
    }
    for (int j = 0; j < W->n; ++j) {
        if (!W->act[j]) continue;
        double m = o_mass(P, W->sp[j]);
        for (int d = 0; d < 3; ++d) W->v[3 * j + d] += 0.5 * dt / m * W->f[3 * j + d];
    }
    I->t += dt;
    I->steps += 1;
    return U;
}

/* ------------------------------------------------------------------------ */
/* Track launch (beam) -- reading: ion at z = -rc, lateral position uniform */
/* in the surface cell at (0,0), direction from tilt and rotation.  Recoil  */
/* (the paper's on-lattice ions with random direction, Sec. 4.1): the ion    */
/* starts on the site of basis atom 0 of cell (0,0,0) of a bulk target with */
/* a direction uniform over the sphere.                                     */
/* ------------------------------------------------------------------------ */
static void o_launch(const o_params* P, uint64_t seed, uint64_t id, o_ion* I)
{
    memset(I, 0, sizeof(*I));
    I->id = id;
    I->primary = id;
    I->key = o_track_key(seed, id);
    uint32_t w[4];
    o_draw(I->key, 0, 0, 0, O_TAG_LAUNCH, w);
    double th, ph;
    if (P->beam_mode == 1) {
        double cmax = cos(P->tilt * O_PI / 180.0);
        double ct = 1.0 - o_unit(w[2]) * (1.0 - cmax);
        th = acos(ct);
        ph = 2.0 * O_PI * o_unit(w[3]);
    } else if (P->beam_mode == 2) {
        /* uniform on the unit sphere: cos(theta) uniform in (-1, 1) */
        th = acos(1.0 - 2.0 * o_unit(w[2]));
        ph = 2.0 * O_PI * o_unit(w[3]);
    } else {
        th = P->tilt * O_PI / 180.0;
        ph = (P->rot_lo + (P->rot_hi - P->rot_lo) * o_unit(w[2])) * O_PI / 180.0;
    }
    double sp = sqrt(2.0 * P->E0 / P->M1);
    if (P->beam_mode == 2) {
        const double(*B)[3] = P->lattice == 1 ? O_FLUORITE : O_DIAMOND;
        for (int d = 0; d < 3; ++d) I->x[d] = B[0][d] * P->a;
    } else {
        I->x[0] = P->a * o_unit(w[0]);
        I->x[1] = P->a * o_unit(w[1]);
        I->x[2] = -P->rc;
    }
    I->v[0] = sp * sin(th) * cos(ph);
    I->v[1] = sp * sin(th) * sin(ph);
    I->v[2] = sp * cos(th);
}

/* exported for tests: the launch state of a primary */
void o_launch_state(const o_params* P, uint64_t seed, uint64_t id, double* x3, double* v3)
{
    o_ion I;
    o_launch(P, seed, id, &I);
    memcpy(x3, I.x, sizeof(I.x));
    memcpy(v3, I.v, sizeof(I.v));
}

static int o_window_capacity(const o_params* P)
{
    return P->n * P->n * P->n * (o_basis_count(P->lattice) > 0 ? o_basis_count(P->lattice) : 1) + 16;
}

/* ------------------------------------------------------------------------ */
/* Tallies                                                                  */
/* ------------------------------------------------------------------------ */
/* Depth of a track for the range tally and the cloning depths: z below the
 * surface; in a bulk target (reading) the distance from the starting site,
 * the range of the paper's recoil runs (Sec. 4.1). */
static double o_depth(const o_params* P, const o_ion* I)
{
    if (P->target != 1) return I->x[2];
    return sqrt(I->x[0] * I->x[0] + I->x[1] * I->x[1] + I->x[2] * I->x[2]);
}

static void o_tally_finish(const o_params* P, o_tally* T, const o_ion* I, int status)
{
    double w = ldexp(1.0, -I->level);
    if (status == O_STOPPED) {
        double z = o_depth(P, I);
        if (z < 0.0) T->hist[P->nbins] += w;
        else {
            double q = floor(z / P->bin_w);
            if (q >= (double)P->nbins) T->hist[P->nbins + 1] += w;
            else T->hist[(int)q] += w;
        }
    } else if (status == O_BACK) {
        T->hist[P->nbins + 2] += w;
    } else {
        T->w_trunc += w;
    }
    T->tracks += 1;
}

/* check the end-of-step state: 0 alive, else a status */
static int o_check(const o_params* P, const o_ion* I)
{
    double E = 0.5 * P->M1 * (I->v[0] * I->v[0] + I->v[1] * I->v[1] + I->v[2] * I->v[2]);
    if (E < P->e_stop) return O_STOPPED;
    if (P->target != 1 && I->x[2] < -P->rc && I->v[2] < 0.0) return O_BACK;
    if (I->steps >= P->step_cap) return O_TRUNC;
    return O_ALIVE;
}

typedef struct {
    o_ion I;
    o_win W;
} o_snap;

/* Run one primary and, depth first, every clone it spawns.  Appends track
 * records (if recs != NULL, up to cap) and tallies. */
typedef struct {
    o_record* r;
    int n, cap;
} o_recbuf;

static void o_recbuf_push(o_recbuf* B, const o_record* R)
{
    if (B->n == B->cap) {
        B->cap = B->cap ? 2 * B->cap : 4;
        B->r = (o_record*)realloc(B->r, sizeof(o_record) * (size_t)B->cap);
    }
    B->r[B->n++] = *R;
}

static int o_run_lineage(const o_params* P, const o_consts* K, uint64_t seed, uint64_t id,
                         o_tally* T, o_recbuf* recs)
{
    int wcap = o_window_capacity(P);
    int depth_cap = P->nthr + 1;
    o_snap* stack = (o_snap*)calloc((size_t)depth_cap, sizeof(o_snap));
    for (int s = 0; s < depth_cap; ++s) o_win_alloc(&stack[s].W, wcap);
    int top = 0;
    o_ion I;
    o_win W;
    o_win_alloc(&W, wcap);
    o_launch(P, seed, id, &I);
    o_window_init(P, &W, &I, I.key);
    o_forces(P, I.x, 1, W.n, W.x, W.sp, I.f, W.f, &I.rho);
    for (;;) {
        int st = O_ALIVE;
        while (st == O_ALIVE) {
            int moved;
            o_step(P, K, &I, &W, I.key, 0.0, 1, &moved, T);
            T->shifts += moved;
            T->steps += 1;
            st = o_check(P, &I);
            if (st != O_ALIVE) break;
            while (I.level < P->nthr && o_depth(P, &I) >= P->thr[I.level]) {
                /* clone: copy of the current state, half weight each */
                I.level += 1;
                o_snap* S = &stack[top++];
                S->I = I;
                S->I.id = o_child_id(I.id, I.level);
                S->I.key = o_track_key(seed, S->I.id);
                o_win_copy(&S->W, &W);
                T->clones += 1;
            }
        }
        o_tally_finish(P, T, &I, st);
        for (int j = 0; j < W.n; ++j)
            if (W.act[j]) o_deposit(P, T, &W.x[3 * j], &W.v[3 * j], P->M2[W.sp[j]], ldexp(1.0, -I.level));
        if (recs) {
            o_record R;
            R.id = I.id; R.primary = I.primary; R.z = o_depth(P, &I); R.t = I.t;
            R.steps = I.steps; R.level = I.level; R.status = st;
            o_recbuf_push(recs, &R);
        }
        if (top == 0) break;
        --top;
        I = stack[top].I;
        o_win_copy(&W, &stack[top].W);
    }
    o_win_free(&W);
    for (int s = 0; s < depth_cap; ++s) o_win_free(&stack[s].W);
    free(stack);
    return 0;
}

static void o_consts_init(const o_params* P, o_consts* K)
{
    K->gam = o_gamma_ls(P);
    K->rho0 = o_rho0(P);
}

/* Run n_ions primaries (ids first_id ... first_id+n_ions-1).  hist has
 * nbins+3 entries (under, over, back appended) and is accumulated into.
 * counters: [steps, tracks, clones, shifts] accumulated; w_trunc added to
 * counters_w[0].  If recs_out is not NULL it receives a malloc'ed array of
 * per-track records (ordered by primary, then depth-first), *nrec its length;
 * release it with o_free. */
int o_run_damage(const o_params* P, int64_t n_ions, int64_t first_id, uint64_t seed, int nthreads,
                 double* hist, int64_t* counters, double* counters_w, o_record** recs_out, int64_t* nrec,
                 double* damage);

int o_run(const o_params* P, int64_t n_ions, int64_t first_id, uint64_t seed, int nthreads,
          double* hist, int64_t* counters, double* counters_w, o_record** recs_out, int64_t* nrec)
{
    return o_run_damage(P, n_ions, first_id, seed, nthreads, hist, counters, counters_w, recs_out, nrec, NULL);
}

/* o_run plus the cumulative damage map (dn^3 voxels + overflow, accumulated
 * into damage when not NULL). */
int o_run_damage(const o_params* P, int64_t n_ions, int64_t first_id, uint64_t seed, int nthreads,
                 double* hist, int64_t* counters, double* counters_w, o_record** recs_out, int64_t* nrec,
                 double* damage)
{
    o_consts K;
    o_consts_init(P, &K);
    int nb = P->nbins + 3;
    size_t nd = (damage && P->dn > 0) ? (size_t)P->dn * P->dn * P->dn + 1 : 0;
    /* damage feedback reads the map as it stood when the run started */
    o_params PF = *P;
    double* snap = NULL;
    if (nd && P->fb_ec > 0.0) {
        snap = (double*)malloc(nd * sizeof(double));
        memcpy(snap, damage, nd * sizeof(double));
        PF.fb_map = snap;
    }
    P = &PF;
    o_recbuf* bufs = recs_out ? (o_recbuf*)calloc((size_t)n_ions, sizeof(o_recbuf)) : NULL;
    int nt = nthreads > 0 ? nthreads : 1;
    double* hs = (double*)calloc((size_t)nt * nb, sizeof(double));
    int64_t* cs = (int64_t*)calloc((size_t)nt * 4, sizeof(int64_t));
    double* ws = (double*)calloc((size_t)nt, sizeof(double));
    double* ds = nd ? (double*)calloc((size_t)nt * nd, sizeof(double)) : NULL;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int64_t i = 0; i < n_ions; ++i) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        o_tally T;
        memset(&T, 0, sizeof(T));
        T.hist = &hs[(size_t)tid * nb];
        T.damage = ds ? &ds[(size_t)tid * nd] : NULL;
        o_run_lineage(P, &K, seed, (uint64_t)(first_id + i), &T, bufs ? &bufs[i] : NULL);
        cs[tid * 4 + 0] += T.steps;
        cs[tid * 4 + 1] += T.tracks;
        cs[tid * 4 + 2] += T.clones;
        cs[tid * 4 + 3] += T.shifts;
        ws[tid] += T.w_trunc;
    }
    for (int t = 0; t < nt; ++t) {
        for (size_t b = 0; b < nd; ++b) damage[b] += ds[(size_t)t * nd + b];
        for (int b = 0; b < nb; ++b) hist[b] += hs[(size_t)t * nb + b];
        for (int c = 0; c < 4; ++c) counters[c] += cs[t * 4 + c];
        counters_w[0] += ws[t];
    }
    if (recs_out) {
        int64_t k = 0;
        for (int64_t i = 0; i < n_ions; ++i) k += bufs[i].n;
        o_record* recs = (o_record*)malloc(sizeof(o_record) * (size_t)(k > 0 ? k : 1));
        k = 0;
        for (int64_t i = 0; i < n_ions; ++i) {
            for (int r = 0; r < bufs[i].n; ++r) recs[k++] = bufs[i].r[r];
            free(bufs[i].r);
        }
        *nrec = k;
        *recs_out = recs;
        free(bufs);
    }
    free(hs);
    free(cs);
    free(ws);
    free(ds);
    free(snap);
    return 0;
}

/* Energy bookkeeping of one primary followed without cloning (for the
 * damage-map balance): out = {E0, final ion KE, final potential energy of
 * the window, energy to electronic stopping, deposited (map + overflow),
 * kinetic energy below the deposit threshold, final window kinetic energy
 * (integrated atoms), steps}. */
int o_track_energy(const o_params* P0, uint64_t seed, uint64_t id, double* out)
{
    o_params P = *P0;
    P.nthr = 0;
    o_consts K;
    o_consts_init(&P, &K);
    size_t nd = (size_t)P.dn * P.dn * P.dn + 1;
    o_tally T;
    memset(&T, 0, sizeof(T));
    double hist_local[1024 + 3];
    if (P.nbins + 3 > 1027 || P.dn <= 0) return -1;
    memset(hist_local, 0, sizeof(hist_local));
    T.hist = hist_local;
    T.damage = (double*)calloc(nd, sizeof(double));
    o_ion I;
    o_win W;
    o_win_alloc(&W, o_window_capacity(&P));
    o_launch(&P, seed, id, &I);
    o_window_init(&P, &W, &I, I.key);
    double U = o_forces(&P, I.x, 1, W.n, W.x, W.sp, I.f, W.f, &I.rho);
    double E0 = 0.5 * P.M1 * (I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2]) + U;
    int st = O_ALIVE;
    while (st == O_ALIVE) {
        int moved;
        U = o_step(&P, &K, &I, &W, I.key, 0.0, 1, &moved, &T);
        st = o_check(&P, &I);
    }
    double ke_win = 0.0;
    for (int j = 0; j < W.n; ++j) {
        if (!W.act[j]) continue;
        ke_win += 0.5 * P.M2[W.sp[j]] *
                  (W.v[3 * j] * W.v[3 * j] + W.v[3 * j + 1] * W.v[3 * j + 1] + W.v[3 * j + 2] * W.v[3 * j + 2]);
    }
    double dep = 0.0;
    for (size_t b = 0; b < nd; ++b) dep += T.damage[b];
    out[0] = E0;
    out[1] = 0.5 * P.M1 * (I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2]);
    out[2] = U;
    out[3] = I.e_elec;
    out[4] = dep;
    out[5] = T.e_dep_sub;
    out[6] = ke_win;
    out[7] = (double)I.steps;
    free(T.damage);
    o_win_free(&W);
    return 0;
}

/* Trajectory of a primary for its first nsteps steps (no cloning): out has
 * 8 doubles per step: x y z t vx vy vz dt.  Also returns the anchor after each
 * step (3 ints) if anchors != NULL.  Returns the number of steps taken. */
int o_trace(const o_params* P, uint64_t seed, uint64_t id, int nsteps, double* out, int* anchors)
{
    o_consts K;
    o_consts_init(P, &K);
    o_ion I;
    o_win W;
    o_win_alloc(&W, o_window_capacity(P));
    o_launch(P, seed, id, &I);
    o_window_init(P, &W, &I, I.key);
    o_forces(P, I.x, 1, W.n, W.x, W.sp, I.f, W.f, &I.rho);
    int s;
    for (s = 0; s < nsteps; ++s) {
        double t0 = I.t;
        int moved;
        o_step(P, &K, &I, &W, I.key, 0.0, 1, &moved, NULL);
        double* o = &out[8 * s];
        o[0] = I.x[0]; o[1] = I.x[1]; o[2] = I.x[2]; o[3] = I.t;
        o[4] = I.v[0]; o[5] = I.v[1]; o[6] = I.v[2]; o[7] = I.t - t0;
        if (anchors) { anchors[3 * s] = W.A[0]; anchors[3 * s + 1] = W.A[1]; anchors[3 * s + 2] = W.A[2]; }
        if (o_check(P, &I) != O_ALIVE) { ++s; break; }
    }
    o_win_free(&W);
    return s;
}

/* Window replay along a prescribed ion path (positions only, no dynamics):
 * after each point, the anchor is written to anchors (3 ints).  At the end
 * the window's atoms are written (cells 3n ints, basis n, xyz 3n) up to cap.
 * Returns the final atom count. */
int o_window_replay(const o_params* P, uint64_t key, int npts, const double* path, int* anchors,
                    int cap, int* cells, int* bas, double* xyz)
{
    o_ion I;
    memset(&I, 0, sizeof(I));
    o_win W;
    o_win_alloc(&W, o_window_capacity(P));
    memcpy(I.x, path, 3 * sizeof(double));
    o_window_init(P, &W, &I, key);
    for (int p = 0; p < npts; ++p) {
        memcpy(I.x, &path[3 * p], 3 * sizeof(double));
        o_window_update(P, &W, &I, key, NULL);
        anchors[3 * p] = W.A[0]; anchors[3 * p + 1] = W.A[1]; anchors[3 * p + 2] = W.A[2];
    }
    int n = W.n;
    for (int j = 0; j < n && j < cap; ++j) {
        for (int d = 0; d < 3; ++d) { cells[3 * j + d] = W.cell[3 * j + d]; xyz[3 * j + d] = W.x[3 * j + d]; }
        bas[j] = W.bas[j];
    }
    o_win_free(&W);
    return n;
}

/* Explicit-atom molecular dynamics (no lattice creation, no window moves):
 * used for two-body scattering and energy-conservation checks.  State is
 * updated in place.  dt_fixed > 0 uses a constant step, else the adaptive
 * rule.  energies (if not NULL) gets nsteps+1 totals (kinetic + potential).
 * Returns the number of steps taken (stops early when the ion-target
 * separation exceeds stop_sep > 0 after having been inside it). */
int o_md_explicit(const o_params* P, double* ion_x, double* ion_v, int n, double* x, double* v,
                  const int* sp, const int* act, int nsteps, double dt_fixed, double stop_sep,
                  double* energies)
{
    o_consts K;
    o_consts_init(P, &K);
    o_ion I;
    memset(&I, 0, sizeof(I));
    memcpy(I.x, ion_x, sizeof(I.x));
    memcpy(I.v, ion_v, sizeof(I.v));
    o_win W;
    o_win_alloc(&W, n + 1);
    W.n = n;
    memcpy(W.x, x, 3 * sizeof(double) * (size_t)n);
    memcpy(W.v, v, 3 * sizeof(double) * (size_t)n);
    memcpy(W.sp, sp, sizeof(int) * (size_t)n);
    memcpy(W.act, act, sizeof(int) * (size_t)n);
    double U = o_forces(P, I.x, 1, W.n, W.x, W.sp, I.f, W.f, &I.rho);
    int inside = 0, s;
    for (s = 0; s <= nsteps; ++s) {
        if (energies) {
            double ke = 0.5 * P->M1 * (I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2]);
            for (int j = 0; j < n; ++j)
                if (W.act[j])
                    ke += 0.5 * o_mass(P, W.sp[j]) *
                          (W.v[3 * j] * W.v[3 * j] + W.v[3 * j + 1] * W.v[3 * j + 1] + W.v[3 * j + 2] * W.v[3 * j + 2]);
            energies[s] = ke + U;
        }
        if (s == nsteps) break;
        int moved;
        U = o_step(P, &K, &I, &W, 0, dt_fixed, 0, &moved, NULL);
        if (0.5 * P->M1 * (I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2]) < P->e_stop) { ++s; break; }
        if (stop_sep > 0.0 && n > 0) {
            double rv[3], r = o_dist(I.x, &W.x[0], rv);
            if (r < stop_sep) inside = 1;
            else if (inside) { ++s; break; }
        }
    }
    memcpy(ion_x, I.x, sizeof(I.x));
    memcpy(ion_v, I.v, sizeof(I.v));
    memcpy(x, W.x, 3 * sizeof(double) * (size_t)n);
    memcpy(v, W.v, 3 * sizeof(double) * (size_t)n);
    o_win_free(&W);
    return s;
}

void o_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Adaptive cloning depths (Sec. 2: depths chosen so that every interval    */
/* between them collects a similar count; re-estimated from all finished    */
/* ions, Sec. 3).  reading: with weights 2^-k the count between d_k and      */
/* d_{k+1} is equal when S(d_k) = 2^-k, S(d) = weighted fraction of          */
/* finished tracks that stopped at depth >= d (backscattered and above-      */
/* surface tracks count as not reaching any d > 0).  S is read off the       */
/* depth histogram with linear interpolation inside a bin.  Targets beyond   */
/* the histogram's last bin give depth +inf (no cloning at that level).      */
/* hist has nbins + 3 entries (under, over, back appended).                  */
/* ------------------------------------------------------------------------ */
int o_update_thresholds(const double* hist, int nbins, double bin_w, int nthr, double* thr)
{
    double total = 0.0;
    for (int b = 0; b < nbins + 3; ++b) total += hist[b];
    if (!(total > 0.0)) return -1;
    double over = hist[nbins + 1];
    for (int k = 1; k <= nthr; ++k) {
        double target = ldexp(total, -k);   /* weight that must lie at or beyond d_k */
        double d = INFINITY;
        if (over < target) {
            /* walk the bins from the deep end: tail(b) = weight at depth >= b*w */
            double tail = over;
            for (int b = nbins - 1; b >= 0; --b) {
                double wb = hist[b];
                if (tail + wb >= target) {
                    /* inside bin b: tail(d) = tail + wb * ((b+1) w - d) / w */
                    double f = (target - tail) / wb;   /* fraction of the bin beyond d */
                    d = (b + 1.0 - f) * bin_w;
                    break;
                }
                tail += wb;
            }
            if (d == INFINITY) d = 0.0;
        }
        thr[k - 1] = d;
    }
    return 0;
}

/* Adaptive run: n_initial primaries without enhancement, then epochs of
 * epoch primaries, the cloning depths re-estimated from the accumulated
 * histogram before each epoch.  The primaries of an epoch run in parallel
 * with the epoch's depths frozen (Sec. 3: a track never sees its depths
 * change).  thr_hist (epochs x 16, may be NULL) receives the depths used by
 * each enhanced epoch; returns the number of enhanced epochs. */
int o_run_adaptive(const o_params* P0, int64_t n_ions, int64_t n_initial, int64_t epoch, uint64_t seed,
                   int nthreads, double* hist, int64_t* counters, double* counters_w, double* thr_hist,
                   int max_epochs)
{
    o_params P = *P0;
    int nthr = P0->nthr;
    int64_t done = 0;
    int ep = 0;
    if (n_initial > n_ions) n_initial = n_ions;
    if (n_initial > 0) {
        P.nthr = 0;
        o_run(&P, n_initial, 0, seed, nthreads, hist, counters, counters_w, NULL, NULL);
        done = n_initial;
    }
    while (done < n_ions) {
        int64_t m = n_ions - done < epoch ? n_ions - done : epoch;
        P.nthr = nthr;
        if (done > 0) {
            double t[16];
            if (o_update_thresholds(hist, P.nbins, P.bin_w, nthr, t) == 0)
                for (int k = 0; k < nthr; ++k) P.thr[k] = t[k];
        }
        if (thr_hist && ep < max_epochs)
            for (int k = 0; k < 16; ++k) thr_hist[16 * ep + k] = k < nthr ? P.thr[k] : 0.0;
        o_run(&P, m, done, seed, nthreads, hist, counters, counters_w, NULL, NULL);
        done += m;
        ++ep;
    }
    return ep;
}

/* Convenience exports for the tests. */
double o_ion_pair_energy(const o_params* P, double Z2, double r, double* dU)
{
    return o_ion_pair(P, Z2, r, dU);
}
double o_taper_export(double r, double rt, double rc, double* dS) { return o_taper(r, rt, rc, dS); }
double o_tau_fs(void) { return O_TAU_FS; }
/* the ZBL-correction basis and correction, exported for the pin tests */
double o_bspline3_export(double u, double* du) { return o_bspline3(u, du); }
double o_spline_corr_export(const double* c, double r, double* dcdr) { return o_spline_corr(c, r, dcdr); }

/* ======================================================================== */
/* Truncated-segment sensitivities (the adjoint workload).                  */
/* reading: the final depth z_T of a track depends on theta = (s_e, s_loc,   */
/* c_1..c_6) only through its last ~200 steps: the state at step s0 =        */
/* 20 floor((T-200)/20) (0 for T < 200) is held fixed, and so are the step   */
/* sizes, the window moves and which side of the surface the ion is on at   */
/* each half kick.  dz_T/dtheta is propagated here by forward-mode tangents */
/* in FP64; tests pin it with central finite differences of the same frozen */
/* replay.                                                                   */
/* ======================================================================== */

static double o_bspline3_d2(double u)
{
    double au = fabs(u);
    if (au >= 2.0) return 0.0;
    if (au >= 1.0) return 2.0 - au;
    return -2.0 + 3.0 * au;
}

/* Ion-target pair U(r) with dU/dr, d2U/dr2 and d(dU/dr)/dc_k (k = 0..5). */
void o_pair_full(const o_params* P, double Z2, double r, double* U, double* dU, double* d2U, double* dUdc)
{
    const double k = P->Z1 * Z2 * O_E2;
    double au = o_zbl_screen_length(P->Z1, Z2);
    double x = r / au, phi = 0.0, dphi = 0.0, d2phi = 0.0;
    for (int i = 0; i < 4; ++i) {
        double e = exp(-O_ZD[i] * x);
        phi += O_ZC[i] * e;
        dphi -= O_ZC[i] * O_ZD[i] * e;
        d2phi += O_ZC[i] * O_ZD[i] * O_ZD[i] * e;
    }
    double V = k * phi / r;
    double V1 = k * (dphi / (au * r) - phi / (r * r));
    double V2 = k * (d2phi / (au * au * r) - 2.0 * dphi / (au * r * r) + 2.0 * phi / (r * r * r));
    /* correction c(r) = sum c_i B_i(u_i), u_i = (ln r - ln r_i)/h */
    double h = (log(O_KNOTS[5]) - log(O_KNOTS[0])) / 5.0;
    double c = 0.0, c1 = 0.0, c2 = 0.0, Bk[6], B1k[6];
    for (int i = 0; i < 6; ++i) {
        double u = (log(r) - log(O_KNOTS[i])) / h, du;
        double b = o_bspline3(u, &du);
        double d2 = o_bspline3_d2(u);
        Bk[i] = b;
        B1k[i] = du / (h * r);                       /* dB_i/dr */
        c += P->spline_c[i] * b;
        c1 += P->spline_c[i] * du / (h * r);
        c2 += P->spline_c[i] * (d2 / (h * h * r * r) - du / (h * r * r));
    }
    double E = exp(c);
    double dS, S = o_taper(r, P->rt, P->rc, &dS);
    double d2S = 0.0;
    if (r > P->rt && r < P->rc) {
        double w = P->rc - P->rt, t = (r - P->rt) / w;
        d2S = (-60.0 * t + 180.0 * t * t - 120.0 * t * t * t) / (w * w);
    }
    *U = V * E * S;
    *dU = V1 * E * S + V * E * c1 * S + V * E * dS;
    *d2U = V2 * E * S + 2.0 * V1 * E * c1 * S + 2.0 * V1 * E * dS + V * E * (c1 * c1 + c2) * S +
           2.0 * V * E * c1 * dS + V * E * d2S;
    for (int i = 0; i < 6; ++i) dUdc[i] = Bk[i] * (*dU) + V * E * S * B1k[i];
}

/* per-step record of the frozen quantities */
typedef struct {
    double dt;
    int A[3];        /* anchor after the step */
    int on1, on2;    /* drag active at the first / second half kick */
} o_segstep;

/* Conservative forces and, for one tangent direction, their derivative:
 * dF = J(x) dx + dF/dtheta_dir.  dir: 0 s_e, 1 s_loc (no effect on F),
 * 2..7 spline c_{dir-2}; dir < 0: no parameter term.  Also returns rho and
 * its gradient contracted with dx (drho), and the d rho/d x_ion, d rho/d x_j
 * needed by the drag. */
static void o_forces_tangent(const o_params* P, const double* xi, int n, const double* x, const int* sp,
                             const double* dxi, const double* dx, int dir, double* fi, double* f, double* dfi,
                             double* df, double* rho, double* drho)
{
    for (int d = 0; d < 3; ++d) { fi[d] = 0.0; dfi[d] = 0.0; }
    for (int j = 0; j < 3 * n; ++j) { f[j] = 0.0; df[j] = 0.0; }
    *rho = 0.0;
    *drho = 0.0;
    for (int j = 0; j < n; ++j) {
        double rv[3], r = o_dist(xi, &x[3 * j], rv);
        if (r >= P->rc) continue;
        double U, dU, d2U, dUdc[6];
        o_pair_full(P, P->Z2[sp[j]], r, &U, &dU, &d2U, dUdc);
        double u[3] = {rv[0] / r, rv[1] / r, rv[2] / r};
        /* relative tangent */
        double q[3] = {dx[3 * j] - dxi[0], dx[3 * j + 1] - dxi[1], dx[3 * j + 2] - dxi[2]};
        double uq = u[0] * q[0] + u[1] * q[1] + u[2] * q[2];
        for (int d = 0; d < 3; ++d) {
            f[3 * j + d] -= dU * u[d];
            fi[d] += dU * u[d];
            /* K q, K = d2U u u^T + (dU/r)(I - u u^T) */
            double Kq = d2U * u[d] * uq + dU / r * (q[d] - u[d] * uq);
            double pth = (dir >= 2) ? dUdc[dir - 2] * u[d] : 0.0;
            df[3 * j + d] -= Kq + pth;
            dfi[d] += Kq + pth;
        }
        double dS, S = o_taper(r, P->rt, P->rc, &dS);
        double e = exp(-r / P->lam_loc);
        *rho += S * e;
        *drho += (dS - S / P->lam_loc) * e * uq;
    }
}

/* Run primary id; record per-step frozen quantities (steps, up to cap).
 * Returns the number of steps T (or -1 if the track did not stop). */
static int64_t o_seg_record(const o_params* P, uint64_t seed, uint64_t id, o_segstep* rec, int64_t cap)
{
    o_params Q = *P;
    Q.nthr = 0;
    o_consts K;
    o_consts_init(&Q, &K);
    o_ion I;
    o_win W;
    o_win_alloc(&W, o_window_capacity(&Q));
    o_launch(&Q, seed, id, &I);
    o_window_init(&Q, &W, &I, I.key);
    o_forces(&Q, I.x, 1, W.n, W.x, W.sp, I.f, W.f, &I.rho);
    int st = O_ALIVE;
    int64_t s = 0;
    while (st == O_ALIVE) {
        int on1 = I.x[2] >= 0.0, moved;
        double t0 = I.t;
        o_step(&Q, &K, &I, &W, I.key, 0.0, 1, &moved, NULL);
        if (s < cap) {
            rec[s].dt = I.t - t0;
            rec[s].A[0] = W.A[0]; rec[s].A[1] = W.A[1]; rec[s].A[2] = W.A[2];
            rec[s].on1 = on1;
            rec[s].on2 = I.x[2] >= 0.0;
        }
        ++s;
        st = o_check(&Q, &I);
    }
    o_win_free(&W);
    return st == O_STOPPED ? s : -1;
}

/* Frozen replay of steps s0..T-1 with parameters Pt (theta may differ from
 * the recording's), optionally with one tangent direction.  The state at s0
 * is produced by re-running the nominal track Pn from its launch.  Returns
 * z_T; *dz gets the tangent dz_T/dtheta_dir (dir >= 0). */
static double o_seg_replay(const o_params* Pn, const o_params* Pt, uint64_t seed, uint64_t id, const o_segstep* rec,
                           int64_t T, int64_t s0, int dir, double* dz)
{
    o_params Qn = *Pn, Qt = *Pt;
    Qn.nthr = Qt.nthr = 0;
    o_consts Kn, Kt;
    o_consts_init(&Qn, &Kn);
    o_consts_init(&Qt, &Kt);
    double g0 = o_gamma_ls(&Qt) / (Qt.s_e != 0.0 ? Qt.s_e : 1.0);   /* gamma without the s_e factor */
    if (Qt.s_e == 0.0) { o_params Q1 = Qt; Q1.s_e = 1.0; g0 = o_gamma_ls(&Q1); }
    double rho0 = o_rho0(&Qt);
    o_ion I;
    o_win W;
    int cap = o_window_capacity(&Qn);
    o_win_alloc(&W, cap);
    o_launch(&Qn, seed, id, &I);
    o_window_init(&Qn, &W, &I, I.key);
    o_forces(&Qn, I.x, 1, W.n, W.x, W.sp, I.f, W.f, &I.rho);
    for (int64_t s = 0; s < s0; ++s) {
        int moved;
        o_step(&Qn, &Kn, &I, &W, I.key, 0.0, 1, &moved, NULL);
    }
    /* tangents (zero at s0: the state there is held fixed); kept per window
     * atom by its (cell, basis) identity through window moves */
    double *dx = (double*)calloc(3 * (size_t)cap, sizeof(double)), *dv = (double*)calloc(3 * (size_t)cap, sizeof(double));
    double *ndx = (double*)calloc(3 * (size_t)cap, sizeof(double)), *ndv = (double*)calloc(3 * (size_t)cap, sizeof(double));
    double dxi[3] = {0, 0, 0}, dvi[3] = {0, 0, 0};
    double *f = (double*)calloc(3 * (size_t)cap, sizeof(double)), *df = (double*)calloc(3 * (size_t)cap, sizeof(double));
    double fi[3], dfi[3], rho, drho;
    /* forces at the start of the segment with the replay's parameters */
    o_forces_tangent(&Qt, I.x, W.n, W.x, W.sp, dxi, dx, dir, fi, f, dfi, df, &rho, &drho);
    for (int64_t s = s0; s < T; ++s) {
        const o_segstep* r = &rec[s];
        double dt = r->dt, h = 0.5 * dt;
        /* --- first half kick with drag at (v, x) */
        double kf = r->on1 ? Qt.s_e * g0 * (1.0 + Qt.s_loc * (rho / rho0 - 1.0)) : 0.0;
        double dk = 0.0;
        if (r->on1 && dir >= 0) {
            dk = Qt.s_e * g0 * Qt.s_loc / rho0 * drho;
            if (dir == 0) dk += g0 * (1.0 + Qt.s_loc * (rho / rho0 - 1.0));
            if (dir == 1) dk += Qt.s_e * g0 * (rho / rho0 - 1.0);
        }
        for (int d = 0; d < 3; ++d) {
            double fe = -kf * I.v[d];
            double dfe = -kf * dvi[d] - dk * I.v[d];
            I.v[d] += h / Qt.M1 * (fi[d] + fe);
            dvi[d] += h / Qt.M1 * (dfi[d] + dfe);
        }
        for (int j = 0; j < W.n; ++j) {
            if (!W.act[j]) continue;
            double m = Qt.M2[W.sp[j]];
            for (int d = 0; d < 3; ++d) {
                W.v[3 * j + d] += h / m * f[3 * j + d];
                dv[3 * j + d] += h / m * df[3 * j + d];
            }
        }
        /* --- drift */
        for (int d = 0; d < 3; ++d) { I.x[d] += dt * I.v[d]; dxi[d] += dt * dvi[d]; }
        for (int j = 0; j < W.n; ++j) {
            if (!W.act[j]) continue;
            for (int d = 0; d < 3; ++d) { W.x[3 * j + d] += dt * W.v[3 * j + d]; dx[3 * j + d] += dt * dv[3 * j + d]; }
        }
        /* --- frozen window move: anchor from the record */
        if (r->A[0] != W.A[0] || r->A[1] != W.A[1] || r->A[2] != W.A[2]) {
            /* remember tangents by atom identity, move the window, restore */
            int n_old = W.n;
            int* ids = (int*)malloc(sizeof(int) * 4 * (size_t)n_old);
            for (int j = 0; j < n_old; ++j) {
                ids[4 * j] = W.cell[3 * j]; ids[4 * j + 1] = W.cell[3 * j + 1]; ids[4 * j + 2] = W.cell[3 * j + 2];
                ids[4 * j + 3] = W.bas[j];
                for (int d = 0; d < 3; ++d) { ndx[3 * j + d] = dx[3 * j + d]; ndv[3 * j + d] = dv[3 * j + d]; }
            }
            o_ion Ia = I;
            Ia.x[0] = (r->A[0] - (Qn.n % 2 == 0 ? 0.5 : 0.0) + 0.5) * Qn.a;   /* a point inside the recorded anchor cell */
            Ia.x[1] = (r->A[1] - (Qn.n % 2 == 0 ? 0.5 : 0.0) + 0.5) * Qn.a;
            Ia.x[2] = (r->A[2] - (Qn.n % 2 == 0 ? 0.5 : 0.0) + 0.5) * Qn.a;
            o_window_update(&Qn, &W, &Ia, I.key, NULL);
            for (int j = 0; j < W.n; ++j) {
                int found = -1;
                for (int q = 0; q < n_old; ++q)
                    if (ids[4 * q] == W.cell[3 * j] && ids[4 * q + 1] == W.cell[3 * j + 1] &&
                        ids[4 * q + 2] == W.cell[3 * j + 2] && ids[4 * q + 3] == W.bas[j]) { found = q; break; }
                for (int d = 0; d < 3; ++d) {
                    dx[3 * j + d] = found >= 0 ? ndx[3 * found + d] : 0.0;
                    dv[3 * j + d] = found >= 0 ? ndv[3 * found + d] : 0.0;
                }
            }
            free(ids);
        }
        /* --- forces at the new positions */
        o_forces_tangent(&Qt, I.x, W.n, W.x, W.sp, dxi, dx, dir, fi, f, dfi, df, &rho, &drho);
        /* --- second half kick with drag at (v_half, x') */
        kf = r->on2 ? Qt.s_e * g0 * (1.0 + Qt.s_loc * (rho / rho0 - 1.0)) : 0.0;
        dk = 0.0;
        if (r->on2 && dir >= 0) {
            dk = Qt.s_e * g0 * Qt.s_loc / rho0 * drho;
            if (dir == 0) dk += g0 * (1.0 + Qt.s_loc * (rho / rho0 - 1.0));
            if (dir == 1) dk += Qt.s_e * g0 * (rho / rho0 - 1.0);
        }
        for (int d = 0; d < 3; ++d) {
            double fe = -kf * I.v[d];
            double dfe = -kf * dvi[d] - dk * I.v[d];
            I.v[d] += h / Qt.M1 * (fi[d] + fe);
            dvi[d] += h / Qt.M1 * (dfi[d] + dfe);
        }
        for (int j = 0; j < W.n; ++j) {
            if (!W.act[j]) continue;
            double m = Qt.M2[W.sp[j]];
            for (int d = 0; d < 3; ++d) {
                W.v[3 * j + d] += h / m * f[3 * j + d];
                dv[3 * j + d] += h / m * df[3 * j + d];
            }
        }
    }
    double z = I.x[2];
    if (dz) *dz = dxi[2];
    free(dx); free(dv); free(ndx); free(ndv); free(f); free(df);
    o_win_free(&W);
    return z;
}

/* Segment sensitivities of primary id: out[0] = z_T, out[1] = T, out[2] =
 * s0, out[3..10] = dz_T/dtheta (forward-mode tangents).  Returns 0, or -1
 * if the track did not stop within cap steps. */
int o_segment_tangent(const o_params* P, uint64_t seed, uint64_t id, int seg, int every, int64_t cap, double* out)
{
    o_segstep* rec = (o_segstep*)calloc((size_t)cap, sizeof(o_segstep));
    int64_t T = o_seg_record(P, seed, id, rec, cap);
    if (T < 0 || T > cap) { free(rec); return -1; }
    int64_t s0 = T > seg ? (int64_t)every * ((T - seg) / every) : 0;
    out[1] = (double)T;
    out[2] = (double)s0;
    for (int dir = 0; dir < 8; ++dir) {
        double dz;
        out[0] = o_seg_replay(P, P, seed, id, rec, T, s0, dir, &dz);
        out[3 + dir] = dz;
    }
    free(rec);
    return 0;
}

/* z_T of the frozen segment replayed with parameter theta_dir changed by
 * delta (for finite differences).  Returns z_T; *T_out, *s0_out set. */
double o_segment_replay_theta(const o_params* P, uint64_t seed, uint64_t id, int seg, int every, int64_t cap, int dir,
                              double delta, int64_t* T_out, int64_t* s0_out)
{
    o_segstep* rec = (o_segstep*)calloc((size_t)cap, sizeof(o_segstep));
    int64_t T = o_seg_record(P, seed, id, rec, cap);
    if (T < 0 || T > cap) { free(rec); return NAN; }
    int64_t s0 = T > seg ? (int64_t)every * ((T - seg) / every) : 0;
    o_params Pt = *P;
    if (dir == 0) Pt.s_e += delta;
    else if (dir == 1) Pt.s_loc += delta;
    else Pt.spline_c[dir - 2] += delta;
    double z = o_seg_replay(P, &Pt, seed, id, rec, T, s0, -1, NULL);
    free(rec);
    *T_out = T;
    *s0_out = s0;
    return z;
}
