/*
 * codonfold_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU oracle for the codon-constrained partition function over a
 * nearest-neighbour secondary-structure model.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the CUDA library
 * never does, and the two share no code, tables or helpers.
 *
 * What it computes (paper, Section "Probability distributions" and
 * Section "Computed quantities"):
 *   Z(psi) = sum over codon sequences c encoding psi and structures s of phi(c)
 *            of  prod_r e^{lw[r][c_r]} * prod_r e^{pb[c_r][c_{r+1}]} * e^{-E(phi(c),s)/RT}
 *   log Z, pair probabilities P_ij (P_ii = unpaired), codon marginals
 *   p_r(c) = d log Z / d lw[r][c], codon-pair marginals d log Z / d pb,
 *   and exact samples of (codon sequence, structure).
 *
 * Arithmetic: C `long double` (x86 80-bit extended, 64-bit significand,
 * 15-bit exponent).  Its range (about e^+-11356) holds Z for sequences of
 * several thousand nucleotides, so the oracle carries NO rescaling logic at
 * all: it is independent of the per-diagonal scaling under test in the CUDA
 * path.  Precision is at least that of binary64.
 *
 * Sequence side: the codon-pair tensor train of the paper (Eq. pair-tt):
 * every position p carries the codon state of its residue r = p/3; the
 * transfer T_p between p and p+1 is the identity inside a residue and
 * e^{lw[r+1][b] + pb[a][b]} across a residue boundary (soft constraints,
 * Section "Incorporating soft constraints").  The train is laid along the
 * backbone of each loop (Section "Dynamic programs over sequences and
 * structures"), so each table entry is a small matrix over the boundary
 * states, i.e. a rectangular block as in Eq. design-fold.
 *
 * Structure side: nearest-neighbour loops.  Energies (kcal/mol):
 *   hairpin (i,j), L=j-i-1>=3      H(L) + tm[x_{i+1}][x_{j-1}],
 *                                   H(L>30) = H(30) + 1.07856 ln(L/30)
 *   stack (i,j),(i+1,j-1)          stack[pt(x_i,x_j)][pt(x_{i+1},x_{j-1})]
 *   bulge, 1 <= L <= 30            Bu(L)
 *   interior l1,l2>=1, L<=30       In(L) + tm[x_{i+1}][x_{j-1}] + tm[x_{l+1}][x_{k-1}]
 *   multiloop, B>=2 branches, U unpaired:
 *                                   a + c(B+1) + bU + d5[x_j][x_{j-1}] + d3[x_i][x_{i+1}]
 *                                   + sum over branches (k,l) d5[x_k][x_{k-1}] + d3[x_l][x_{l+1}]
 *   exterior branch (k,l)          d5[x_k][x_{k-1}] (k>0) + d3[x_l][x_{l+1}] (l<n-1)
 * Hairpins need >= 3 unpaired bases (Section "Dynamic programming algorithms
 * for fixed RNA sequences": B_{i,j} = 0 for |j-i| < 4).
 *
 * Multiloop and exterior tables carry a "port" per end: (codon state, type)
 * with type U (the end base is unpaired) or P (the end base is the paired
 * end of a branch).  The backbone transition X_p between p and p+1 is T_p
 * times the 3' dangle of a branch ending at p (type P at p) and the 5' dangle
 * of a branch starting at p+1 (type P at p+1).
 *
 * Recursions (all i <= j, d = j - i), plain and in this order per cell:
 *   C[i][j]   = T_i C[i+1][j]                        (chain, C[i][i] = I)
 *   QB[i][j]  = ok(i,j) * ( T_i ((S o TMo) ) T_{j-1} + stack + bulges + ML )
 *               S = eH(d-1) C[i+1][j-1] + sum_{interior k,l} eIn C[i+1][k-1] XI[k][l] C[l+1][j-1]
 *               ML = ea ec X_i[(a,P),:] QM2[i+1][j-1] X_{j-1}[:,(b,P)]
 *   XI[k][l]  = (T_{k-1} QB[k][l] T_l) o TMi           (inner pair seen from its loop)
 *   QM1[i][j] = one branch starting at i: ec QB[i][j] (port P at j)
 *               + sum_l ec eb^{j-l} QB[i][l] X_l[P->U] C[l+1][j] (port U at j)
 *   QM[i][j]  = >= 1 branch: QM1[i][j] (port P at i)
 *               + sum_k (UN(i,k-1) + QM[i][k-1]) X_{k-1}[->P] QM1[k][j]
 *   QM2[i][j] = >= 2 branches: sum_k QM[i][k-1] X_{k-1}[->P] QM1[k][j]
 *   Q5[j]     = exterior prefix [0..j]: Q5[j-1] X_{j-1}[->U]
 *               + (P cols) QB[0][j] + sum_k Q5[k-1] X_{k-1}[->P] QB[k][j]
 *   Z         = sum_a u0[a] sum_port Q5[n-1][a][port]
 * The outside pass is the reverse-mode adjoint of exactly these statements,
 * written by hand; the sampler is a stochastic traceback over the same
 * tables.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long double R;

#define NS 6   /* maximum codon states of one residue */
#define NPT 12 /* ports: state a with type t at index a + 6 t; t = 0 U, 1 P */
#define MAXLOOP 30
#define TU 0
#define TP 1

/* Standard genetic code, codons in lexicographic order over A,C,G,U. */
static const char *OR_CODE64 =
    "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF";
static const char *OR_AA = "ARNDCQEGHILKMFPSTWYV";

typedef struct {
  int n, m;
  int any_pair; /* test hook: every base pairs with every base, pair type 0 */
  R kT;
  R est[6][6], eHl[MAXLOOP + 1], eBu[MAXLOOP + 1], eIn[MAXLOOP + 1];
  R etm[4][4], ed5[4][4], ed3[4][4];
  R Hlast, ea, eb, ec;
  int *M;             /* [n] states per position */
  int (*base)[NS];    /* [n][NS] base of state a at position p */
  int (*cid)[NS];     /* [n][NS] sense codon id of state a */
  R (*T)[NS][NS];     /* [n] transfer p -> p+1 (last unused) */
  R (*X)[NPT][NPT];   /* [n] typed transition p -> p+1 */
  R u0[NS];
  const unsigned char *allow; /* optional n*n pair mask, 0 forbids (i,j) */
  /* inside tables, triangular cell index */
  R (*C)[NS][NS];
  R (*QB)[NS][NS];
  R (*XI)[NS][NS];
  R (*QM1)[NS][NPT];
  R (*QM)[NPT][NPT];
  R (*QM2)[NPT][NPT];
  R (*Q5)[NS][NPT];
  R Z;
  /* adjoints */
  R (*hC)[NS][NS];
  R (*hQB)[NS][NS];
  R (*hXI)[NS][NS];
  R (*hQM1)[NS][NPT];
  R (*hQM)[NPT][NPT];
  R (*hQM2)[NPT][NPT];
  R (*hQ5)[NS][NPT];
  R (*hT)[NS][NS];
  R (*hX)[NPT][NPT];
  R hu0[NS];
} octx;

static inline size_t tri(const octx *c, int i, int j) {
  return (size_t)i * c->n - (size_t)i * (i - 1) / 2 + (size_t)(j - i);
}

static inline R bz(const octx *c, double e) { return expl(-(R)e / c->kT); }

static int pair_type(int x, int y) {
  /* AU, CG, GC, UA, GU, UG -> 0..5; -1 otherwise */
  if (x == 0 && y == 3) return 0;
  if (x == 1 && y == 2) return 1;
  if (x == 2 && y == 1) return 2;
  if (x == 3 && y == 0) return 3;
  if (x == 2 && y == 3) return 4;
  if (x == 3 && y == 2) return 5;
  return -1;
}

static int codon_base(int codon64, int k) { return (codon64 >> (2 * (2 - k))) & 3; }

static int sense_id(int codon64) {
  int id = 0;
  for (int c = 0; c < codon64; c++)
    if (OR_CODE64[c] != '*') id++;
  return id;
}

/* Hairpin Boltzmann factor without the mismatch term. */
static R eH(const octx *c, int L) {
  if (L <= MAXLOOP) return c->eHl[L];
  return expl(-(c->Hlast + (R)1.07856 * logl((R)L / (R)MAXLOOP)) / c->kT);
}

static int pairable(const octx *c, int i, int a, int j, int b) {
  if (j - i < 4) return 0;
  if (c->allow && !c->allow[(size_t)i * c->n + j]) return 0;
  if (c->any_pair) return 1;
  return pair_type(c->base[i][a], c->base[j][b]) >= 0;
}

static R stackf(const octx *c, int i, int a, int j, int b, int a2, int b2) {
  if (c->any_pair) return c->est[0][0];
  int o = pair_type(c->base[i][a], c->base[j][b]);
  int in = pair_type(c->base[i + 1][a2], c->base[j - 1][b2]);
  if (o < 0 || in < 0) return 0;
  return c->est[o][in];
}

/* ---------------------------------------------------------------- setup */

static void free_ctx(octx *c) {
  free(c->M); free(c->base); free(c->cid); free(c->T); free(c->X);
  free(c->C); free(c->QB); free(c->XI); free(c->QM1); free(c->QM); free(c->QM2); free(c->Q5);
  free(c->hC); free(c->hQB); free(c->hXI); free(c->hQM1); free(c->hQM); free(c->hQM2);
  free(c->hQ5); free(c->hT); free(c->hX);
  memset(c, 0, sizeof(*c));
}

static int setup(octx *c, const double *params, const int *res, int m, const double *lw,
                 const double *pb, const unsigned char *allow, int any_pair) {
  memset(c, 0, sizeof(*c));
  c->m = m;
  c->n = 3 * m;
  c->any_pair = any_pair;
  c->allow = allow;
  int n = c->n;
  const double *st = params, *H = params + 36, *Bu = params + 67, *In = params + 98;
  const double *tm = params + 129, *d5 = params + 145, *d3 = params + 161;
  double tempC = params[180];
  c->kT = (R)1.98717e-3L * ((R)tempC + (R)273.15L);
  for (int x = 0; x < 6; x++)
    for (int y = 0; y < 6; y++) c->est[x][y] = bz(c, st[6 * x + y]);
  for (int L = 0; L <= MAXLOOP; L++) {
    c->eHl[L] = bz(c, H[L]);
    c->eBu[L] = bz(c, Bu[L]);
    c->eIn[L] = bz(c, In[L]);
  }
  c->Hlast = (R)H[MAXLOOP];
  for (int x = 0; x < 4; x++)
    for (int y = 0; y < 4; y++) {
      c->etm[x][y] = bz(c, tm[4 * x + y]);
      c->ed5[x][y] = bz(c, d5[4 * x + y]);
      c->ed3[x][y] = bz(c, d3[4 * x + y]);
    }
  c->ea = bz(c, params[177]);
  c->eb = bz(c, params[178]);
  c->ec = bz(c, params[179]);

  c->M = calloc(n, sizeof(int));
  c->base = calloc(n, sizeof(*c->base));
  c->cid = calloc(n, sizeof(*c->cid));
  c->T = calloc(n, sizeof(*c->T));
  c->X = calloc(n, sizeof(*c->X));
  for (int r = 0; r < m; r++) {
    if (res[r] < 0 || res[r] >= 20) return -1;
    char aa = OR_AA[res[r]];
    int cnt = 0, cods[NS];
    for (int k = 0; k < 64; k++)
      if (OR_CODE64[k] == aa) cods[cnt++] = k;
    for (int off = 0; off < 3; off++) {
      int p = 3 * r + off;
      c->M[p] = cnt;
      for (int a = 0; a < cnt; a++) {
        c->base[p][a] = codon_base(cods[a], off);
        c->cid[p][a] = sense_id(cods[a]);
      }
    }
  }
  for (int p = 0; p + 1 < n; p++) {
    int r1 = (p + 1) / 3;
    for (int a = 0; a < c->M[p]; a++)
      for (int b = 0; b < c->M[p + 1]; b++) {
        if (p % 3 != 2) {
          c->T[p][a][b] = (a == b) ? 1 : 0;
        } else {
          double w = lw ? lw[6 * r1 + b] : 0.0;
          if (pb) w += pb[61 * c->cid[p][a] + c->cid[p + 1][b]];
          c->T[p][a][b] = expl((R)w);
        }
      }
    /* typed transition */
    for (int a = 0; a < c->M[p]; a++)
      for (int b = 0; b < c->M[p + 1]; b++)
        for (int t = 0; t < 2; t++)
          for (int t2 = 0; t2 < 2; t2++) {
            R f = c->T[p][a][b];
            int x = c->base[p][a], y = c->base[p + 1][b];
            if (t == TP) f *= c->ed3[x][y];
            if (t2 == TP) f *= c->ed5[y][x];
            c->X[p][a + 6 * t][b + 6 * t2] = f;
          }
  }
  for (int a = 0; a < c->M[0]; a++) c->u0[a] = expl((R)(lw ? lw[a] : 0.0));
  size_t ncell = (size_t)n * (n + 1) / 2;
  c->C = calloc(ncell, sizeof(*c->C));
  c->QB = calloc(ncell, sizeof(*c->QB));
  c->XI = calloc(ncell, sizeof(*c->XI));
  c->QM1 = calloc(ncell, sizeof(*c->QM1));
  c->QM = calloc(ncell, sizeof(*c->QM));
  c->QM2 = calloc(ncell, sizeof(*c->QM2));
  c->Q5 = calloc(n, sizeof(*c->Q5));
  if (!c->C || !c->QB || !c->XI || !c->QM1 || !c->QM || !c->QM2 || !c->Q5) return -2;
  return 0;
}

/* port index lists of position p: states only, or (state, type) */
static int ports_of(const octx *c, int p, int *out) {
  int k = 0;
  for (int t = 0; t < 2; t++)
    for (int a = 0; a < c->M[p]; a++) out[k++] = a + 6 * t;
  return k;
}

/* ---------------------------------------------------------------- inside */

/* S block of the loop closed by (i,j): hairpin + interior loops, before the
 * outer mismatch and the outer transfers are applied.  M_{i+1} x M_{j-1}. */
static void inner_sum(const octx *c, int i, int j, R S[NS][NS]) {
  int x = i + 1, y = j - 1;
  memset(S, 0, sizeof(R) * NS * NS);
  R h = eH(c, j - i - 1);
  const R(*Ch)[NS] = c->C[tri(c, x, y)];
  for (int u = 0; u < c->M[x]; u++)
    for (int v = 0; v < c->M[y]; v++) S[u][v] = h * Ch[u][v];
  for (int l1 = 1; l1 <= MAXLOOP; l1++)
    for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++) {
      int k = i + 1 + l1, l = j - 1 - l2;
      if (l - k < 4) continue;
      R w = c->eIn[l1 + l2];
      const R(*C1)[NS] = c->C[tri(c, x, k - 1)];
      const R(*XI)[NS] = c->XI[tri(c, k, l)];
      const R(*C2)[NS] = c->C[tri(c, l + 1, y)];
      R tmp[NS][NS] = {{0}};
      for (int u = 0; u < c->M[x]; u++)
        for (int w2 = 0; w2 < c->M[k - 1]; w2++) {
          R a = C1[u][w2];
          if (a == 0) continue;
          for (int z = 0; z < c->M[l + 1]; z++) tmp[u][z] += a * XI[w2][z];
        }
      for (int u = 0; u < c->M[x]; u++)
        for (int z = 0; z < c->M[l + 1]; z++) {
          R a = w * tmp[u][z];
          if (a == 0) continue;
          for (int v = 0; v < c->M[y]; v++) S[u][v] += a * C2[z][v];
        }
    }
}

static R tmo(const octx *c, int x, int u, int y, int v) {
  if (c->any_pair) return c->etm[0][0];
  return c->etm[c->base[x][u]][c->base[y][v]];
}

static void cell_chain(octx *c, int i, int j) {
  R(*Cij)[NS] = c->C[tri(c, i, j)];
  if (i == j) {
    for (int a = 0; a < c->M[i]; a++) Cij[a][a] = 1;
    return;
  }
  const R(*Cn)[NS] = c->C[tri(c, i + 1, j)];
  for (int a = 0; a < c->M[i]; a++)
    for (int s = 0; s < c->M[i + 1]; s++) {
      R t = c->T[i][a][s];
      if (t == 0) continue;
      for (int b = 0; b < c->M[j]; b++) Cij[a][b] += t * Cn[s][b];
    }
}

static void cell_qb(octx *c, int i, int j) {
  int n = c->n;
  (void)n;
  R acc[NS][NS] = {{0}};
  int Mi = c->M[i], Mj = c->M[j], Mx = c->M[i + 1], My = c->M[j - 1];
  /* hairpin + interior: T_i (S o TMo) T_{j-1} */
  R S[NS][NS];
  inner_sum(c, i, j, S);
  R K[NS][NS] = {{0}};
  for (int u = 0; u < Mx; u++)
    for (int v = 0; v < My; v++) K[u][v] = S[u][v] * tmo(c, i + 1, u, j - 1, v);
  R KT[NS][NS] = {{0}};
  for (int u = 0; u < Mx; u++)
    for (int v = 0; v < My; v++)
      for (int b = 0; b < Mj; b++) KT[u][b] += K[u][v] * c->T[j - 1][v][b];
  for (int a = 0; a < Mi; a++)
    for (int u = 0; u < Mx; u++)
      for (int b = 0; b < Mj; b++) acc[a][b] += c->T[i][a][u] * KT[u][b];
  /* stack */
  if (j - i - 2 >= 4) {
    const R(*Qin)[NS] = c->QB[tri(c, i + 1, j - 1)];
    for (int a = 0; a < Mi; a++)
      for (int b = 0; b < Mj; b++)
        for (int a2 = 0; a2 < Mx; a2++)
          for (int b2 = 0; b2 < My; b2++) {
            R q = Qin[a2][b2];
            if (q == 0) continue;
            acc[a][b] += c->T[i][a][a2] * q * c->T[j - 1][b2][b] * stackf(c, i, a, j, b, a2, b2);
          }
  }
  /* bulges */
  for (int L = 1; L <= MAXLOOP; L++) {
    /* 3' side bulge: inner pair (i+1, l), l = j-1-L */
    int l = j - 1 - L;
    if (l - (i + 1) >= 4) {
      const R(*Q)[NS] = c->QB[tri(c, i + 1, l)];
      const R(*Cr)[NS] = c->C[tri(c, l, j)];
      R t1[NS][NS] = {{0}};
      for (int a = 0; a < Mi; a++)
        for (int a2 = 0; a2 < Mx; a2++) {
          R t = c->T[i][a][a2];
          if (t == 0) continue;
          for (int s = 0; s < c->M[l]; s++) t1[a][s] += t * Q[a2][s];
        }
      for (int a = 0; a < Mi; a++)
        for (int s = 0; s < c->M[l]; s++)
          for (int b = 0; b < Mj; b++) acc[a][b] += c->eBu[L] * t1[a][s] * Cr[s][b];
    }
    /* 5' side bulge: inner pair (k, j-1), k = i+1+L */
    int k = i + 1 + L;
    if ((j - 1) - k >= 4) {
      const R(*Q)[NS] = c->QB[tri(c, k, j - 1)];
      const R(*Cl)[NS] = c->C[tri(c, i, k)];
      R t1[NS][NS] = {{0}};
      for (int a = 0; a < Mi; a++)
        for (int s = 0; s < c->M[k]; s++) {
          R t = Cl[a][s];
          if (t == 0) continue;
          for (int b2 = 0; b2 < My; b2++) t1[a][b2] += t * Q[s][b2];
        }
      for (int a = 0; a < Mi; a++)
        for (int b2 = 0; b2 < My; b2++)
          for (int b = 0; b < Mj; b++) acc[a][b] += c->eBu[L] * t1[a][b2] * c->T[j - 1][b2][b];
    }
  }
  /* multiloop closed by (i,j) */
  if (j - i - 2 >= 9) {
    const R(*Q2)[NPT] = c->QM2[tri(c, i + 1, j - 1)];
    int px[NPT], py[NPT];
    int nx = ports_of(c, i + 1, px), ny = ports_of(c, j - 1, py);
    R w = c->ea * c->ec;
    for (int a = 0; a < Mi; a++) {
      R row[NPT] = {0}; /* X_i[(a,P)][p] QM2[p][q] */
      for (int pi = 0; pi < nx; pi++) {
        R xa = c->X[i][a + 6][px[pi]];
        if (xa == 0) continue;
        for (int qi = 0; qi < ny; qi++) row[py[qi]] += xa * Q2[px[pi]][py[qi]];
      }
      for (int b = 0; b < Mj; b++) {
        R s = 0;
        for (int qi = 0; qi < ny; qi++) s += row[py[qi]] * c->X[j - 1][py[qi]][b + 6];
        acc[a][b] += w * s;
      }
    }
  }
  R(*QB)[NS] = c->QB[tri(c, i, j)];
  for (int a = 0; a < Mi; a++)
    for (int b = 0; b < Mj; b++) QB[a][b] = pairable(c, i, a, j, b) ? acc[a][b] : 0;
}

static R tmi(const octx *c, int k, int w, int l, int z) {
  /* inner mismatch of pair (k,l) seen from its enclosing loop: tm[x_{l+1}][x_{k-1}] */
  if (c->any_pair) return c->etm[0][0];
  return c->etm[c->base[l + 1][z]][c->base[k - 1][w]];
}

static void cell_xi(octx *c, int k, int l) {
  if (k < 1 || l > c->n - 2) return;
  const R(*Q)[NS] = c->QB[tri(c, k, l)];
  R(*XI)[NS] = c->XI[tri(c, k, l)];
  R t1[NS][NS] = {{0}};
  for (int w = 0; w < c->M[k - 1]; w++)
    for (int a = 0; a < c->M[k]; a++)
      for (int b = 0; b < c->M[l]; b++) t1[w][b] += c->T[k - 1][w][a] * Q[a][b];
  for (int w = 0; w < c->M[k - 1]; w++)
    for (int z = 0; z < c->M[l + 1]; z++) {
      R s = 0;
      for (int b = 0; b < c->M[l]; b++) s += t1[w][b] * c->T[l][b][z];
      XI[w][z] = s * tmi(c, k, w, l, z);
    }
}

static void cell_qm1(octx *c, int i, int j) {
  R(*Q1)[NPT] = c->QM1[tri(c, i, j)];
  const R(*QB)[NS] = c->QB[tri(c, i, j)];
  for (int a = 0; a < c->M[i]; a++)
    for (int b = 0; b < c->M[j]; b++) Q1[a][b + 6] = c->ec * QB[a][b];
  for (int l = i + 4; l <= j - 1; l++) {
    const R(*Q)[NS] = c->QB[tri(c, i, l)];
    const R(*Cr)[NS] = c->C[tri(c, l + 1, j)];
    R w = c->ec * powl(c->eb, (R)(j - l));
    R t1[NS][NS] = {{0}}; /* QB[i][l] X_l[P->U] */
    for (int a = 0; a < c->M[i]; a++)
      for (int s = 0; s < c->M[l]; s++) {
        R q = Q[a][s];
        if (q == 0) continue;
        for (int e = 0; e < c->M[l + 1]; e++) t1[a][e] += q * c->X[l][s + 6][e];
      }
    for (int a = 0; a < c->M[i]; a++)
      for (int e = 0; e < c->M[l + 1]; e++) {
        R t = w * t1[a][e];
        if (t == 0) continue;
        for (int b = 0; b < c->M[j]; b++) Q1[a][b] += t * Cr[e][b];
      }
  }
}

/* out[pr][b] (b = state at k) = sum_q L[pr][q] X_{k-1}[q][(b,P)] */
static void left_to_P(const octx *c, int k, const R L[NPT][NPT], const int *pr, int npr,
                      R out[NPT][NS]) {
  int pq[NPT];
  int nq = ports_of(c, k - 1, pq);
  for (int ri = 0; ri < npr; ri++)
    for (int b = 0; b < c->M[k]; b++) {
      R s = 0;
      for (int qi = 0; qi < nq; qi++) s += L[pr[ri]][pq[qi]] * c->X[k - 1][pq[qi]][b + 6];
      out[pr[ri]][b] = s;
    }
}

static void cell_qm(octx *c, int i, int j) {
  R(*QM)[NPT] = c->QM[tri(c, i, j)];
  const R(*Q1)[NPT] = c->QM1[tri(c, i, j)];
  int pi_[NPT], pj[NPT];
  int ni = ports_of(c, i, pi_), nj = ports_of(c, j, pj);
  for (int a = 0; a < c->M[i]; a++)
    for (int qi = 0; qi < nj; qi++) QM[a + 6][pj[qi]] += Q1[a][pj[qi]];
  for (int k = i + 1; k <= j - 4; k++) {
    R L[NPT][NPT] = {{0}};
    const R(*Qp)[NPT] = c->QM[tri(c, i, k - 1)];
    for (int ri = 0; ri < ni; ri++)
      for (int qi = 0; qi < 2 * c->M[k - 1]; qi++) {
        int q = (qi < c->M[k - 1]) ? qi : qi - c->M[k - 1] + 6;
        L[pi_[ri]][q] = Qp[pi_[ri]][q];
      }
    R un = powl(c->eb, (R)(k - i));
    const R(*Cu)[NS] = c->C[tri(c, i, k - 1)];
    for (int a = 0; a < c->M[i]; a++)
      for (int s = 0; s < c->M[k - 1]; s++) L[a][s] += un * Cu[a][s];
    R LX[NPT][NS];
    left_to_P(c, k, (const R(*)[NPT])L, pi_, ni, LX);
    const R(*Qk)[NPT] = c->QM1[tri(c, k, j)];
    for (int ri = 0; ri < ni; ri++)
      for (int b = 0; b < c->M[k]; b++) {
        R t = LX[pi_[ri]][b];
        if (t == 0) continue;
        for (int qi = 0; qi < nj; qi++) QM[pi_[ri]][pj[qi]] += t * Qk[b][pj[qi]];
      }
  }
}

static void cell_qm2(octx *c, int i, int j) {
  R(*Q2)[NPT] = c->QM2[tri(c, i, j)];
  int pi_[NPT], pj[NPT];
  int ni = ports_of(c, i, pi_), nj = ports_of(c, j, pj);
  for (int k = i + 5; k <= j - 4; k++) {
    const R(*Qp)[NPT] = c->QM[tri(c, i, k - 1)];
    R LX[NPT][NS];
    left_to_P(c, k, Qp, pi_, ni, LX);
    const R(*Qk)[NPT] = c->QM1[tri(c, k, j)];
    for (int ri = 0; ri < ni; ri++)
      for (int b = 0; b < c->M[k]; b++) {
        R t = LX[pi_[ri]][b];
        if (t == 0) continue;
        for (int qi = 0; qi < nj; qi++) Q2[pi_[ri]][pj[qi]] += t * Qk[b][pj[qi]];
      }
  }
}

static void exterior(octx *c) {
  int n = c->n;
  for (int a = 0; a < c->M[0]; a++) c->Q5[0][a][a] = 1;
  for (int j = 1; j < n; j++) {
    R(*Q)[NPT] = c->Q5[j];
    int pp[NPT];
    int np = ports_of(c, j - 1, pp);
    for (int a = 0; a < c->M[0]; a++)
      for (int b = 0; b < c->M[j]; b++) {
        R s = 0;
        for (int qi = 0; qi < np; qi++) s += c->Q5[j - 1][a][pp[qi]] * c->X[j - 1][pp[qi]][b];
        Q[a][b] = s;
      }
    const R(*QB0)[NS] = c->QB[tri(c, 0, j)];
    for (int a = 0; a < c->M[0]; a++)
      for (int b = 0; b < c->M[j]; b++) Q[a][b + 6] += QB0[a][b];
    for (int k = 1; k <= j - 4; k++) {
      int pq[NPT];
      int nq = ports_of(c, k - 1, pq);
      const R(*QBk)[NS] = c->QB[tri(c, k, j)];
      for (int a = 0; a < c->M[0]; a++) {
        R w[NS] = {0};
        for (int s = 0; s < c->M[k]; s++)
          for (int qi = 0; qi < nq; qi++)
            w[s] += c->Q5[k - 1][a][pq[qi]] * c->X[k - 1][pq[qi]][s + 6];
        for (int b = 0; b < c->M[j]; b++) {
          R t = 0;
          for (int s = 0; s < c->M[k]; s++) t += w[s] * QBk[s][b];
          Q[a][b + 6] += t;
        }
      }
    }
  }
  R Z = 0;
  int pp[NPT];
  int np = ports_of(c, n - 1, pp);
  for (int a = 0; a < c->M[0]; a++)
    for (int qi = 0; qi < np; qi++) Z += c->u0[a] * c->Q5[n - 1][a][pp[qi]];
  c->Z = Z;
}

static void inside(octx *c) {
  int n = c->n;
  for (int d = 0; d < n; d++) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n - d; i++) {
      int j = i + d;
      cell_chain(c, i, j);
      if (d >= 4) {
        cell_qb(c, i, j);
        cell_xi(c, i, j);
        cell_qm1(c, i, j);
        cell_qm(c, i, j);
        if (d >= 9) cell_qm2(c, i, j);
      }
    }
  }
  exterior(c);
}

/* ---------------------------------------------------------------- outside */
/* Reverse-mode adjoint of every statement of the inside pass, in reverse
 * order.  hX = dZ/dX etc.  Accumulation is sequential (scatter form). */

static int alloc_adjoint(octx *c) {
  int n = c->n;
  size_t ncell = (size_t)n * (n + 1) / 2;
  c->hC = calloc(ncell, sizeof(*c->hC));
  c->hQB = calloc(ncell, sizeof(*c->hQB));
  c->hXI = calloc(ncell, sizeof(*c->hXI));
  c->hQM1 = calloc(ncell, sizeof(*c->hQM1));
  c->hQM = calloc(ncell, sizeof(*c->hQM));
  c->hQM2 = calloc(ncell, sizeof(*c->hQM2));
  c->hQ5 = calloc(n, sizeof(*c->hQ5));
  c->hT = calloc(n, sizeof(*c->hT));
  c->hX = calloc(n, sizeof(*c->hX));
  if (!c->hC || !c->hQB || !c->hXI || !c->hQM1 || !c->hQM || !c->hQM2 || !c->hQ5 || !c->hT ||
      !c->hX)
    return -2;
  return 0;
}

static void exterior_adj(octx *c) {
  int n = c->n;
  int pp[NPT];
  int np = ports_of(c, n - 1, pp);
  for (int a = 0; a < c->M[0]; a++) {
    R s = 0;
    for (int qi = 0; qi < np; qi++) {
      s += c->Q5[n - 1][a][pp[qi]];
      c->hQ5[n - 1][a][pp[qi]] = c->u0[a];
    }
    c->hu0[a] = s;
  }
  for (int j = n - 1; j >= 1; j--) {
    R(*hQ)[NPT] = c->hQ5[j];
    /* pairs closing at j */
    R(*hB0)[NS] = c->hQB[tri(c, 0, j)];
    for (int a = 0; a < c->M[0]; a++)
      for (int b = 0; b < c->M[j]; b++) hB0[a][b] += hQ[a][b + 6];
    for (int k = 1; k <= j - 4; k++) {
      int pq[NPT];
      int nq = ports_of(c, k - 1, pq);
      const R(*QBk)[NS] = c->QB[tri(c, k, j)];
      R(*hQBk)[NS] = c->hQB[tri(c, k, j)];
      for (int a = 0; a < c->M[0]; a++) {
        R w[NS] = {0};
        for (int s = 0; s < c->M[k]; s++)
          for (int qi = 0; qi < nq; qi++)
            w[s] += c->Q5[k - 1][a][pq[qi]] * c->X[k - 1][pq[qi]][s + 6];
        R hw[NS] = {0};
        for (int s = 0; s < c->M[k]; s++)
          for (int b = 0; b < c->M[j]; b++) {
            hQBk[s][b] += w[s] * hQ[a][b + 6];
            hw[s] += hQ[a][b + 6] * QBk[s][b];
          }
        for (int s = 0; s < c->M[k]; s++)
          for (int qi = 0; qi < nq; qi++) {
            c->hQ5[k - 1][a][pq[qi]] += hw[s] * c->X[k - 1][pq[qi]][s + 6];
            c->hX[k - 1][pq[qi]][s + 6] += c->Q5[k - 1][a][pq[qi]] * hw[s];
          }
      }
    }
    /* unpaired j */
    int pj1[NPT];
    int nj1 = ports_of(c, j - 1, pj1);
    for (int a = 0; a < c->M[0]; a++)
      for (int b = 0; b < c->M[j]; b++) {
        R g = hQ[a][b];
        if (g == 0) continue;
        for (int qi = 0; qi < nj1; qi++) {
          c->hQ5[j - 1][a][pj1[qi]] += g * c->X[j - 1][pj1[qi]][b];
          c->hX[j - 1][pj1[qi]][b] += c->Q5[j - 1][a][pj1[qi]] * g;
        }
      }
  }
}

static void cell_qm2_adj(octx *c, int i, int j) {
  const R(*hQ2)[NPT] = c->hQM2[tri(c, i, j)];
  int pi_[NPT], pj[NPT];
  int ni = ports_of(c, i, pi_), nj = ports_of(c, j, pj);
  for (int k = i + 5; k <= j - 4; k++) {
    const R(*Qp)[NPT] = c->QM[tri(c, i, k - 1)];
    R(*hQp)[NPT] = c->hQM[tri(c, i, k - 1)];
    const R(*Qk)[NPT] = c->QM1[tri(c, k, j)];
    R(*hQk)[NPT] = c->hQM1[tri(c, k, j)];
    R LX[NPT][NS];
    left_to_P(c, k, Qp, pi_, ni, LX);
    R hLX[NPT][NS] = {{0}};
    for (int ri = 0; ri < ni; ri++)
      for (int b = 0; b < c->M[k]; b++)
        for (int qi = 0; qi < nj; qi++) {
          R g = hQ2[pi_[ri]][pj[qi]];
          hQk[b][pj[qi]] += LX[pi_[ri]][b] * g;
          hLX[pi_[ri]][b] += g * Qk[b][pj[qi]];
        }
    int pq[NPT];
    int nq = ports_of(c, k - 1, pq);
    for (int ri = 0; ri < ni; ri++)
      for (int b = 0; b < c->M[k]; b++) {
        R g = hLX[pi_[ri]][b];
        if (g == 0) continue;
        for (int qi = 0; qi < nq; qi++) {
          hQp[pi_[ri]][pq[qi]] += g * c->X[k - 1][pq[qi]][b + 6];
          c->hX[k - 1][pq[qi]][b + 6] += Qp[pi_[ri]][pq[qi]] * g;
        }
      }
  }
}

static void cell_qm_adj(octx *c, int i, int j) {
  const R(*hQM)[NPT] = c->hQM[tri(c, i, j)];
  R(*hQ1)[NPT] = c->hQM1[tri(c, i, j)];
  int pi_[NPT], pj[NPT];
  int ni = ports_of(c, i, pi_), nj = ports_of(c, j, pj);
  for (int a = 0; a < c->M[i]; a++)
    for (int qi = 0; qi < nj; qi++) hQ1[a][pj[qi]] += hQM[a + 6][pj[qi]];
  for (int k = i + 1; k <= j - 4; k++) {
    R L[NPT][NPT] = {{0}};
    const R(*Qp)[NPT] = c->QM[tri(c, i, k - 1)];
    R(*hQp)[NPT] = c->hQM[tri(c, i, k - 1)];
    int pq[NPT];
    int nq = ports_of(c, k - 1, pq);
    for (int ri = 0; ri < ni; ri++)
      for (int qi = 0; qi < nq; qi++) L[pi_[ri]][pq[qi]] = Qp[pi_[ri]][pq[qi]];
    R un = powl(c->eb, (R)(k - i));
    const R(*Cu)[NS] = c->C[tri(c, i, k - 1)];
    R(*hCu)[NS] = c->hC[tri(c, i, k - 1)];
    for (int a = 0; a < c->M[i]; a++)
      for (int s = 0; s < c->M[k - 1]; s++) L[a][s] += un * Cu[a][s];
    R LX[NPT][NS];
    left_to_P(c, k, (const R(*)[NPT])L, pi_, ni, LX);
    const R(*Qk)[NPT] = c->QM1[tri(c, k, j)];
    R(*hQk)[NPT] = c->hQM1[tri(c, k, j)];
    R hLX[NPT][NS] = {{0}};
    for (int ri = 0; ri < ni; ri++)
      for (int b = 0; b < c->M[k]; b++)
        for (int qi = 0; qi < nj; qi++) {
          R g = hQM[pi_[ri]][pj[qi]];
          hQk[b][pj[qi]] += LX[pi_[ri]][b] * g;
          hLX[pi_[ri]][b] += g * Qk[b][pj[qi]];
        }
    for (int ri = 0; ri < ni; ri++)
      for (int b = 0; b < c->M[k]; b++) {
        R g = hLX[pi_[ri]][b];
        if (g == 0) continue;
        for (int qi = 0; qi < nq; qi++) {
          R hl = g * c->X[k - 1][pq[qi]][b + 6];
          hQp[pi_[ri]][pq[qi]] += hl;
          int p = pi_[ri], q = pq[qi];
          if (p < 6 && q < 6) hCu[p][q] += un * hl;
          c->hX[k - 1][pq[qi]][b + 6] += L[pi_[ri]][pq[qi]] * g;
        }
      }
  }
}

static void cell_qm1_adj(octx *c, int i, int j) {
  const R(*hQ1)[NPT] = c->hQM1[tri(c, i, j)];
  R(*hQB)[NS] = c->hQB[tri(c, i, j)];
  for (int a = 0; a < c->M[i]; a++)
    for (int b = 0; b < c->M[j]; b++) hQB[a][b] += c->ec * hQ1[a][b + 6];
  for (int l = i + 4; l <= j - 1; l++) {
    const R(*Q)[NS] = c->QB[tri(c, i, l)];
    R(*hQ)[NS] = c->hQB[tri(c, i, l)];
    const R(*Cr)[NS] = c->C[tri(c, l + 1, j)];
    R(*hCr)[NS] = c->hC[tri(c, l + 1, j)];
    R w = c->ec * powl(c->eb, (R)(j - l));
    /* V[s][b] = sum_e X_l[(s,P)][(e,U)] Cr[e][b] */
    R V[NS][NS] = {{0}};
    for (int s = 0; s < c->M[l]; s++)
      for (int e = 0; e < c->M[l + 1]; e++)
        for (int b = 0; b < c->M[j]; b++) V[s][b] += c->X[l][s + 6][e] * Cr[e][b];
    /* hQ[a][s] += w sum_b hQ1[a][b] V[s][b]; hB[s][b] = w sum_a Q[a][s] hQ1[a][b] */
    R hB[NS][NS] = {{0}};
    for (int a = 0; a < c->M[i]; a++)
      for (int b = 0; b < c->M[j]; b++) {
        R g = w * hQ1[a][b];
        if (g == 0) continue;
        for (int s = 0; s < c->M[l]; s++) {
          hQ[a][s] += g * V[s][b];
          hB[s][b] += Q[a][s] * g;
        }
      }
    for (int s = 0; s < c->M[l]; s++)
      for (int e = 0; e < c->M[l + 1]; e++)
        for (int b = 0; b < c->M[j]; b++) {
          c->hX[l][s + 6][e] += hB[s][b] * Cr[e][b];
          hCr[e][b] += c->X[l][s + 6][e] * hB[s][b];
        }
  }
}

static void cell_xi_adj(octx *c, int k, int l) {
  if (k < 1 || l > c->n - 2) return;
  const R(*Q)[NS] = c->QB[tri(c, k, l)];
  R(*hQ)[NS] = c->hQB[tri(c, k, l)];
  const R(*hXI)[NS] = c->hXI[tri(c, k, l)];
  R G[NS][NS] = {{0}};
  for (int w = 0; w < c->M[k - 1]; w++)
    for (int z = 0; z < c->M[l + 1]; z++) G[w][z] = hXI[w][z] * tmi(c, k, w, l, z);
  for (int w = 0; w < c->M[k - 1]; w++)
    for (int a = 0; a < c->M[k]; a++)
      for (int b = 0; b < c->M[l]; b++)
        for (int z = 0; z < c->M[l + 1]; z++) {
          R g = G[w][z];
          if (g == 0) continue;
          R tl = c->T[k - 1][w][a], tr = c->T[l][b][z];
          c->hT[k - 1][w][a] += g * Q[a][b] * tr;
          hQ[a][b] += g * tl * tr;
          c->hT[l][b][z] += g * tl * Q[a][b];
        }
}

static void cell_qb_adj(octx *c, int i, int j) {
  int Mi = c->M[i], Mj = c->M[j], Mx = c->M[i + 1], My = c->M[j - 1];
  const R(*hQB)[NS] = c->hQB[tri(c, i, j)];
  R G[NS][NS] = {{0}};
  int any = 0;
  for (int a = 0; a < Mi; a++)
    for (int b = 0; b < Mj; b++)
      if (pairable(c, i, a, j, b)) {
        G[a][b] = hQB[a][b];
        if (G[a][b] != 0) any = 1;
      }
  if (!any) return;
  /* hairpin + interior */
  R S[NS][NS];
  inner_sum(c, i, j, S);
  R K[NS][NS] = {{0}}, TM[NS][NS] = {{0}};
  for (int u = 0; u < Mx; u++)
    for (int v = 0; v < My; v++) {
      TM[u][v] = tmo(c, i + 1, u, j - 1, v);
      K[u][v] = S[u][v] * TM[u][v];
    }
  R hS[NS][NS] = {{0}};
  for (int a = 0; a < Mi; a++)
    for (int b = 0; b < Mj; b++) {
      R g = G[a][b];
      if (g == 0) continue;
      for (int u = 0; u < Mx; u++)
        for (int v = 0; v < My; v++) {
          R tl = c->T[i][a][u], tr = c->T[j - 1][v][b];
          c->hT[i][a][u] += g * K[u][v] * tr;
          c->hT[j - 1][v][b] += g * tl * K[u][v];
          hS[u][v] += g * tl * tr * TM[u][v];
        }
    }
  {
    int x = i + 1, y = j - 1;
    R h = eH(c, j - i - 1);
    R(*hCh)[NS] = c->hC[tri(c, x, y)];
    for (int u = 0; u < Mx; u++)
      for (int v = 0; v < My; v++) hCh[u][v] += h * hS[u][v];
    for (int l1 = 1; l1 <= MAXLOOP; l1++)
      for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++) {
        int k = i + 1 + l1, l = j - 1 - l2;
        if (l - k < 4) continue;
        R w = c->eIn[l1 + l2];
        const R(*C1)[NS] = c->C[tri(c, x, k - 1)];
        const R(*XI)[NS] = c->XI[tri(c, k, l)];
        const R(*C2)[NS] = c->C[tri(c, l + 1, y)];
        R(*hC1)[NS] = c->hC[tri(c, x, k - 1)];
        R(*hXI)[NS] = c->hXI[tri(c, k, l)];
        R(*hC2)[NS] = c->hC[tri(c, l + 1, y)];
        int Mw = c->M[k - 1], Mz = c->M[l + 1];
        /* A = XI C2 (Mw x My), B = C1 XI (Mx x Mz), D = hS C2^T (Mx x Mz) */
        R A[NS][NS] = {{0}}, B[NS][NS] = {{0}}, D[NS][NS] = {{0}};
        for (int w2 = 0; w2 < Mw; w2++)
          for (int z = 0; z < Mz; z++)
            for (int v = 0; v < My; v++) A[w2][v] += XI[w2][z] * C2[z][v];
        for (int u = 0; u < Mx; u++)
          for (int w2 = 0; w2 < Mw; w2++)
            for (int z = 0; z < Mz; z++) B[u][z] += C1[u][w2] * XI[w2][z];
        for (int u = 0; u < Mx; u++)
          for (int z = 0; z < Mz; z++)
            for (int v = 0; v < My; v++) D[u][z] += hS[u][v] * C2[z][v];
        for (int u = 0; u < Mx; u++)
          for (int w2 = 0; w2 < Mw; w2++) {
            R s = 0;
            for (int v = 0; v < My; v++) s += hS[u][v] * A[w2][v];
            hC1[u][w2] += w * s;
          }
        for (int w2 = 0; w2 < Mw; w2++)
          for (int z = 0; z < Mz; z++) {
            R s = 0;
            for (int u = 0; u < Mx; u++) s += C1[u][w2] * D[u][z];
            hXI[w2][z] += w * s;
          }
        for (int z = 0; z < Mz; z++)
          for (int v = 0; v < My; v++) {
            R s = 0;
            for (int u = 0; u < Mx; u++) s += B[u][z] * hS[u][v];
            hC2[z][v] += w * s;
          }
      }
  }
  /* stack */
  if (j - i - 2 >= 4) {
    const R(*Qin)[NS] = c->QB[tri(c, i + 1, j - 1)];
    R(*hQin)[NS] = c->hQB[tri(c, i + 1, j - 1)];
    for (int a = 0; a < Mi; a++)
      for (int b = 0; b < Mj; b++) {
        R g = G[a][b];
        if (g == 0) continue;
        for (int a2 = 0; a2 < Mx; a2++)
          for (int b2 = 0; b2 < My; b2++) {
            R e = stackf(c, i, a, j, b, a2, b2) * g;
            if (e == 0) continue;
            R tl = c->T[i][a][a2], tr = c->T[j - 1][b2][b], q = Qin[a2][b2];
            c->hT[i][a][a2] += e * q * tr;
            hQin[a2][b2] += e * tl * tr;
            c->hT[j - 1][b2][b] += e * tl * q;
          }
      }
  }
  /* bulges */
  for (int L = 1; L <= MAXLOOP; L++) {
    R w = c->eBu[L];
    int l = j - 1 - L;
    if (l - (i + 1) >= 4) {
      const R(*Q)[NS] = c->QB[tri(c, i + 1, l)];
      R(*hQ)[NS] = c->hQB[tri(c, i + 1, l)];
      const R(*Cr)[NS] = c->C[tri(c, l, j)];
      R(*hCr)[NS] = c->hC[tri(c, l, j)];
      int Ml = c->M[l];
      R QC[NS][NS] = {{0}}, TQ[NS][NS] = {{0}};
      for (int a2 = 0; a2 < Mx; a2++)
        for (int s = 0; s < Ml; s++)
          for (int b = 0; b < Mj; b++) QC[a2][b] += Q[a2][s] * Cr[s][b];
      for (int a = 0; a < Mi; a++)
        for (int a2 = 0; a2 < Mx; a2++)
          for (int s = 0; s < Ml; s++) TQ[a][s] += c->T[i][a][a2] * Q[a2][s];
      for (int a = 0; a < Mi; a++)
        for (int b = 0; b < Mj; b++) {
          R g = w * G[a][b];
          if (g == 0) continue;
          for (int a2 = 0; a2 < Mx; a2++) c->hT[i][a][a2] += g * QC[a2][b];
          for (int s = 0; s < Ml; s++) hCr[s][b] += TQ[a][s] * g;
          for (int a2 = 0; a2 < Mx; a2++) {
            R t = g * c->T[i][a][a2];
            if (t == 0) continue;
            for (int s = 0; s < Ml; s++) hQ[a2][s] += t * Cr[s][b];
          }
        }
    }
    int k = i + 1 + L;
    if ((j - 1) - k >= 4) {
      const R(*Q)[NS] = c->QB[tri(c, k, j - 1)];
      R(*hQ)[NS] = c->hQB[tri(c, k, j - 1)];
      const R(*Cl)[NS] = c->C[tri(c, i, k)];
      R(*hCl)[NS] = c->hC[tri(c, i, k)];
      int Mk = c->M[k];
      R QT[NS][NS] = {{0}}, CQ[NS][NS] = {{0}};
      for (int s = 0; s < Mk; s++)
        for (int b2 = 0; b2 < My; b2++)
          for (int b = 0; b < Mj; b++) QT[s][b] += Q[s][b2] * c->T[j - 1][b2][b];
      for (int a = 0; a < Mi; a++)
        for (int s = 0; s < Mk; s++)
          for (int b2 = 0; b2 < My; b2++) CQ[a][b2] += Cl[a][s] * Q[s][b2];
      for (int a = 0; a < Mi; a++)
        for (int b = 0; b < Mj; b++) {
          R g = w * G[a][b];
          if (g == 0) continue;
          for (int s = 0; s < Mk; s++) hCl[a][s] += g * QT[s][b];
          for (int b2 = 0; b2 < My; b2++) c->hT[j - 1][b2][b] += CQ[a][b2] * g;
          for (int s = 0; s < Mk; s++) {
            R t = g * Cl[a][s];
            if (t == 0) continue;
            for (int b2 = 0; b2 < My; b2++) hQ[s][b2] += t * c->T[j - 1][b2][b];
          }
        }
    }
  }
  /* multiloop */
  if (j - i - 2 >= 9) {
    const R(*Q2)[NPT] = c->QM2[tri(c, i + 1, j - 1)];
    R(*hQ2)[NPT] = c->hQM2[tri(c, i + 1, j - 1)];
    int px[NPT], py[NPT];
    int nx = ports_of(c, i + 1, px), ny = ports_of(c, j - 1, py);
    R w = c->ea * c->ec;
    for (int a = 0; a < Mi; a++)
      for (int b = 0; b < Mj; b++) {
        R g = w * G[a][b];
        if (g == 0) continue;
        for (int pi = 0; pi < nx; pi++)
          for (int qi = 0; qi < ny; qi++) {
            int p = px[pi], q = py[qi];
            R xa = c->X[i][a + 6][p], xb = c->X[j - 1][q][b + 6];
            c->hX[i][a + 6][p] += g * Q2[p][q] * xb;
            hQ2[p][q] += g * xa * xb;
            c->hX[j - 1][q][b + 6] += g * xa * Q2[p][q];
          }
      }
  }
}

static void cell_chain_adj(octx *c, int i, int j) {
  if (i == j) return;
  const R(*hC)[NS] = c->hC[tri(c, i, j)];
  const R(*Cn)[NS] = c->C[tri(c, i + 1, j)];
  R(*hCn)[NS] = c->hC[tri(c, i + 1, j)];
  for (int a = 0; a < c->M[i]; a++)
    for (int s = 0; s < c->M[i + 1]; s++)
      for (int b = 0; b < c->M[j]; b++) {
        c->hT[i][a][s] += hC[a][b] * Cn[s][b];
        hCn[s][b] += c->T[i][a][s] * hC[a][b];
      }
}

static void outside(octx *c) {
  int n = c->n;
  exterior_adj(c);
  for (int d = n - 1; d >= 0; d--)
    for (int i = 0; i + d < n; i++) {
      int j = i + d;
      if (d >= 4) {
        if (d >= 9) cell_qm2_adj(c, i, j);
        cell_qm_adj(c, i, j);
        cell_qm1_adj(c, i, j);
        cell_xi_adj(c, i, j);
        cell_qb_adj(c, i, j);
      }
      cell_chain_adj(c, i, j);
    }
  /* typed transitions back onto the transfers */
  for (int p = 0; p + 1 < n; p++)
    for (int a = 0; a < c->M[p]; a++)
      for (int b = 0; b < c->M[p + 1]; b++)
        for (int t = 0; t < 2; t++)
          for (int t2 = 0; t2 < 2; t2++) {
            int x = c->base[p][a], y = c->base[p + 1][b];
            R f = 1;
            if (t == TP) f *= c->ed3[x][y];
            if (t2 == TP) f *= c->ed5[y][x];
            c->hT[p][a][b] += c->hX[p][a + 6 * t][b + 6 * t2] * f;
          }
}

/* ---------------------------------------------------------------- API */

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

int or_inside(const double *params, const int *res, int m, const double *lw, const double *pb,
              const unsigned char *allow, int any_pair, double *logZ) {
  if (m < 1) return OR_EINVAL;
  octx c;
  int rc = setup(&c, params, res, m, lw, pb, allow, any_pair);
  if (rc) {
    free_ctx(&c);
    return rc == -1 ? OR_EINVAL : OR_ENOMEM;
  }
  inside(&c);
  *logZ = (double)logl(c.Z);
  free_ctx(&c);
  return OR_OK;
}

/* Outputs (any may be NULL):
 *  P[n*n]      pair probabilities, P[i*n+i] = unpaired probability
 *  pcod[m*6]   codon marginals by state slot (codon-id order within the residue)
 *  ppair[61*61] d log Z / d pb (codon-pair marginals summed over residue boundaries)
 *  ptrans[(m-1)*36] joint codon marginals of each adjacent residue pair [r][a][b]
 */
int or_outside(const double *params, const int *res, int m, const double *lw, const double *pb,
               const unsigned char *allow, int any_pair, double *logZ, double *P, double *pcod,
               double *ppair, double *ptrans) {
  if (m < 1) return OR_EINVAL;
  octx c;
  int rc = setup(&c, params, res, m, lw, pb, allow, any_pair);
  if (rc) {
    free_ctx(&c);
    return rc == -1 ? OR_EINVAL : OR_ENOMEM;
  }
  inside(&c);
  *logZ = (double)logl(c.Z);
  if (alloc_adjoint(&c)) {
    free_ctx(&c);
    return OR_ENOMEM;
  }
  outside(&c);
  int n = c.n;
  R Z = c.Z;
  if (P) {
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) P[(size_t)i * n + j] = 0;
    for (int i = 0; i < n; i++)
      for (int j = i + 4; j < n; j++) {
        R s = 0;
        const R(*Q)[NS] = c.QB[tri(&c, i, j)];
        const R(*hQ)[NS] = c.hQB[tri(&c, i, j)];
        for (int a = 0; a < c.M[i]; a++)
          for (int b = 0; b < c.M[j]; b++) s += Q[a][b] * hQ[a][b];
        P[(size_t)i * n + j] = P[(size_t)j * n + i] = (double)(s / Z);
      }
    for (int i = 0; i < n; i++) {
      R s = 0;
      for (int j = 0; j < n; j++)
        if (j != i) s += P[(size_t)i * n + j];
      P[(size_t)i * n + i] = (double)(1 - s);
    }
  }
  if (pcod) {
    for (int k = 0; k < 6 * m; k++) pcod[k] = 0;
    /* the first transfer of each residue lies inside the residue: its
     * diagonal carries the residue's codon marginal */
    for (int r = 0; r < m; r++) {
      int p = 3 * r;
      for (int a = 0; a < c.M[p]; a++) pcod[6 * r + a] = (double)(c.T[p][a][a] * c.hT[p][a][a] / Z);
    }
  }
  if (ppair) {
    for (int k = 0; k < 61 * 61; k++) ppair[k] = 0;
    for (int r = 0; r + 1 < m; r++) {
      int p = 3 * r + 2;
      for (int a = 0; a < c.M[p]; a++)
        for (int b = 0; b < c.M[p + 1]; b++)
          ppair[61 * c.cid[p][a] + c.cid[p + 1][b]] += (double)(c.T[p][a][b] * c.hT[p][a][b] / Z);
    }
  }
  if (ptrans) {
    for (int r = 0; r + 1 < m; r++) {
      int p = 3 * r + 2;
      for (int a = 0; a < 6; a++)
        for (int b = 0; b < 6; b++) {
          double v = 0;
          if (a < c.M[p] && b < c.M[p + 1]) v = (double)(c.T[p][a][b] * c.hT[p][a][b] / Z);
          ptrans[36 * r + 6 * a + b] = v;
        }
    }
  }
  free_ctx(&c);
  return OR_OK;
}

/* ---------------------------------------------------------------- sampler */
/* Stochastic traceback over the inside tables.  Each step draws one uniform
 * u in [0,1) and takes the first alternative (in the fixed enumeration order
 * written in each routine) whose running sum exceeds u * total.  Random
 * numbers come from SplitMix64 (Steele, Lea & Flood 2014), one stream per
 * sample seeded with seed + 0x9E3779B97F4A7C15 * (sample + 1). */

typedef struct {
  uint64_t s;
} sm64;

static uint64_t sm64_next(sm64 *g) {
  uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static R sm64_unif(sm64 *g) { return (R)(sm64_next(g) >> 11) * (R)(1.0 / 9007199254740992.0); }

typedef struct {
  octx *c;
  sm64 g;
  int *state;   /* [n] sampled state per position */
  int *partner; /* [n] */
  int err;
} strace;

/* choose index among w[0..k) */
static int pick(strace *t, const R *w, int k) {
  R tot = 0;
  for (int q = 0; q < k; q++) tot += w[q];
  if (!(tot > 0)) {
    t->err = 1;
    return 0;
  }
  R u = sm64_unif(&t->g) * tot, acc = 0;
  int last = 0;
  for (int q = 0; q < k; q++) {
    if (w[q] <= 0) continue;
    acc += w[q];
    last = q;
    if (u < acc) return q;
  }
  return last;
}

static void set_state(strace *t, int p, int a) {
  if (t->state[p] >= 0 && t->state[p] != a) t->err = 2;
  t->state[p] = a;
}

/* Unpaired-or-not chain x..y with fixed end states: sample the states of the
 * positions strictly between (bridge over the transfer matrices). */
static void tb_chain(strace *t, int x, int y, int a, int b) {
  octx *c = t->c;
  set_state(t, x, a);
  int cur = a;
  for (int p = x; p < y; p++) {
    R w[NS];
    const R(*Cn)[NS] = c->C[tri(c, p + 1, y)];
    for (int s = 0; s < c->M[p + 1]; s++) w[s] = c->T[p][cur][s] * Cn[s][b];
    cur = pick(t, w, c->M[p + 1]);
    set_state(t, p + 1, cur);
  }
  if (cur != b) t->err = 3;
}

static void tb_qb(strace *t, int i, int j, int a, int b);
static void tb_qm(strace *t, int i, int j, int p1, int p2);
static void tb_qm1(strace *t, int i, int j, int a, int p2);

static void tb_qm2(strace *t, int i, int j, int p1, int p2) {
  octx *c = t->c;
  /* alternatives: (k, q at k-1, s at k) in order k asc, q port order, s asc */
  int cnt = 0;
  for (int k = i + 5; k <= j - 4; k++) cnt += 2 * c->M[k - 1] * c->M[k];
  R *w = malloc(sizeof(R) * (cnt > 0 ? cnt : 1));
  int idx = 0;
  for (int k = i + 5; k <= j - 4; k++) {
    const R(*Qp)[NPT] = c->QM[tri(c, i, k - 1)];
    const R(*Qk)[NPT] = c->QM1[tri(c, k, j)];
    int pq[NPT];
    int nq = ports_of(c, k - 1, pq);
    for (int qi = 0; qi < nq; qi++)
      for (int s = 0; s < c->M[k]; s++)
        w[idx++] = Qp[p1][pq[qi]] * c->X[k - 1][pq[qi]][s + 6] * Qk[s][p2];
  }
  int q = pick(t, w, cnt);
  free(w);
  idx = 0;
  for (int k = i + 5; k <= j - 4; k++) {
    int pq[NPT];
    int nq = ports_of(c, k - 1, pq);
    int span = nq * c->M[k];
    if (q < idx + span) {
      int r = q - idx;
      int qp = pq[r / c->M[k]], s = r % c->M[k];
      tb_qm(t, i, k - 1, p1, qp);
      tb_qm1(t, k, j, s, p2);
      return;
    }
    idx += span;
  }
}

static void tb_qm(strace *t, int i, int j, int p1, int p2) {
  octx *c = t->c;
  /* alternatives: [k=i branch] then for k=i+1..j-4: (unpaired-prefix or QM, q, s) */
  int cnt = 1;
  for (int k = i + 1; k <= j - 4; k++) cnt += 2 * (2 * c->M[k - 1]) * c->M[k];
  R *w = malloc(sizeof(R) * cnt);
  int idx = 0;
  w[idx++] = (p1 >= 6) ? c->QM1[tri(c, i, j)][p1 - 6][p2] : 0;
  for (int k = i + 1; k <= j - 4; k++) {
    const R(*Qp)[NPT] = c->QM[tri(c, i, k - 1)];
    const R(*Cu)[NS] = c->C[tri(c, i, k - 1)];
    const R(*Qk)[NPT] = c->QM1[tri(c, k, j)];
    R un = powl(c->eb, (R)(k - i));
    int pq[NPT];
    int nq = ports_of(c, k - 1, pq);
    for (int kind = 0; kind < 2; kind++)
      for (int qi = 0; qi < nq; qi++)
        for (int s = 0; s < c->M[k]; s++) {
          R l;
          if (kind == 0) l = (p1 < 6 && pq[qi] < 6) ? un * Cu[p1][pq[qi]] : 0;
          else l = Qp[p1][pq[qi]];
          w[idx++] = l * c->X[k - 1][pq[qi]][s + 6] * Qk[s][p2];
        }
  }
  int q = pick(t, w, cnt);
  free(w);
  if (q == 0) {
    tb_qm1(t, i, j, p1 - 6, p2);
    return;
  }
  idx = 1;
  for (int k = i + 1; k <= j - 4; k++) {
    int pq[NPT];
    int nq = ports_of(c, k - 1, pq);
    int span = 2 * nq * c->M[k];
    if (q < idx + span) {
      int r = q - idx;
      int kind = r / (nq * c->M[k]);
      r %= nq * c->M[k];
      int qp = pq[r / c->M[k]], s = r % c->M[k];
      if (kind == 0) {
        tb_chain(t, i, k - 1, p1, qp);
      } else {
        tb_qm(t, i, k - 1, p1, qp);
      }
      tb_qm1(t, k, j, s, p2);
      return;
    }
    idx += span;
  }
}

static void tb_qm1(strace *t, int i, int j, int a, int p2) {
  octx *c = t->c;
  if (p2 >= 6) {
    tb_qb(t, i, j, a, p2 - 6);
    return;
  }
  int b = p2;
  /* alternatives: (l, s at l, e at l+1) */
  int cnt = 0;
  for (int l = i + 4; l <= j - 1; l++) cnt += c->M[l] * c->M[l + 1];
  R *w = malloc(sizeof(R) * (cnt > 0 ? cnt : 1));
  int idx = 0;
  for (int l = i + 4; l <= j - 1; l++) {
    const R(*Q)[NS] = c->QB[tri(c, i, l)];
    const R(*Cr)[NS] = c->C[tri(c, l + 1, j)];
    R wl = c->ec * powl(c->eb, (R)(j - l));
    for (int s = 0; s < c->M[l]; s++)
      for (int e = 0; e < c->M[l + 1]; e++) w[idx++] = wl * Q[a][s] * c->X[l][s + 6][e] * Cr[e][b];
  }
  int q = pick(t, w, cnt);
  free(w);
  idx = 0;
  for (int l = i + 4; l <= j - 1; l++) {
    int span = c->M[l] * c->M[l + 1];
    if (q < idx + span) {
      int r = q - idx;
      int s = r / c->M[l + 1], e = r % c->M[l + 1];
      tb_qb(t, i, l, a, s);
      tb_chain(t, l + 1, j, e, b);
      return;
    }
    idx += span;
  }
}

static void tb_qb(strace *t, int i, int j, int a, int b) {
  octx *c = t->c;
  int Mi = c->M[i], Mj = c->M[j], Mx = c->M[i + 1], My = c->M[j - 1];
  (void)Mi;
  (void)Mj;
  t->partner[i] = j;
  t->partner[j] = i;
  set_state(t, i, a);
  set_state(t, j, b);
  /* Level 1 alternatives: 0 hairpin, 1 stack, 2..61 bulges (3' then 5' per L),
   * then interior (l1,l2) in loop order, then multiloop. */
  int nint = 0;
  for (int l1 = 1; l1 <= MAXLOOP; l1++)
    for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++) nint++;
  int nalt = 2 + 2 * MAXLOOP + nint + 1;
  R *w = calloc(nalt, sizeof(R));
  int x = i + 1, y = j - 1;
  /* hairpin */
  {
    R h = eH(c, j - i - 1);
    const R(*Ch)[NS] = c->C[tri(c, x, y)];
    R s = 0;
    for (int u = 0; u < Mx; u++)
      for (int v = 0; v < My; v++)
        s += c->T[i][a][u] * h * Ch[u][v] * tmo(c, x, u, y, v) * c->T[j - 1][v][b];
    w[0] = s;
  }
  if (j - i - 2 >= 4) {
    const R(*Qin)[NS] = c->QB[tri(c, x, y)];
    R s = 0;
    for (int a2 = 0; a2 < Mx; a2++)
      for (int b2 = 0; b2 < My; b2++)
        s += c->T[i][a][a2] * Qin[a2][b2] * c->T[j - 1][b2][b] * stackf(c, i, a, j, b, a2, b2);
    w[1] = s;
  }
  for (int L = 1; L <= MAXLOOP; L++) {
    int l = j - 1 - L;
    if (l - x >= 4) {
      const R(*Q)[NS] = c->QB[tri(c, x, l)];
      const R(*Cr)[NS] = c->C[tri(c, l, j)];
      R s = 0;
      for (int a2 = 0; a2 < Mx; a2++)
        for (int e = 0; e < c->M[l]; e++) s += c->T[i][a][a2] * Q[a2][e] * Cr[e][b];
      w[2 + 2 * (L - 1)] = c->eBu[L] * s;
    }
    int k = i + 1 + L;
    if (y - k >= 4) {
      const R(*Q)[NS] = c->QB[tri(c, k, y)];
      const R(*Cl)[NS] = c->C[tri(c, i, k)];
      R s = 0;
      for (int e = 0; e < c->M[k]; e++)
        for (int b2 = 0; b2 < My; b2++) s += Cl[a][e] * Q[e][b2] * c->T[j - 1][b2][b];
      w[3 + 2 * (L - 1)] = c->eBu[L] * s;
    }
  }
  int idx = 2 + 2 * MAXLOOP;
  for (int l1 = 1; l1 <= MAXLOOP; l1++)
    for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++, idx++) {
      int k = i + 1 + l1, l = j - 1 - l2;
      if (l - k < 4) continue;
      const R(*C1)[NS] = c->C[tri(c, x, k - 1)];
      const R(*XI)[NS] = c->XI[tri(c, k, l)];
      const R(*C2)[NS] = c->C[tri(c, l + 1, y)];
      R s = 0;
      for (int u = 0; u < Mx; u++)
        for (int v = 0; v < My; v++) {
          R tt = c->T[i][a][u] * tmo(c, x, u, y, v) * c->T[j - 1][v][b];
          if (tt == 0) continue;
          R inner = 0;
          for (int w2 = 0; w2 < c->M[k - 1]; w2++)
            for (int z = 0; z < c->M[l + 1]; z++) inner += C1[u][w2] * XI[w2][z] * C2[z][v];
          s += tt * inner;
        }
      w[idx] = c->eIn[l1 + l2] * s;
    }
  if (j - i - 2 >= 9) {
    const R(*Q2)[NPT] = c->QM2[tri(c, x, y)];
    int px[NPT], py[NPT];
    int nx = ports_of(c, x, px), ny = ports_of(c, y, py);
    R s = 0;
    for (int pi = 0; pi < nx; pi++)
      for (int qi = 0; qi < ny; qi++)
        s += c->X[i][a + 6][px[pi]] * Q2[px[pi]][py[qi]] * c->X[j - 1][py[qi]][b + 6];
    w[nalt - 1] = c->ea * c->ec * s;
  }
  int q = pick(t, w, nalt);
  free(w);
  if (q == 0) {
    R h = eH(c, j - i - 1);
    const R(*Ch)[NS] = c->C[tri(c, x, y)];
    R ww[NS * NS];
    for (int u = 0; u < Mx; u++)
      for (int v = 0; v < My; v++)
        ww[u * My + v] = c->T[i][a][u] * h * Ch[u][v] * tmo(c, x, u, y, v) * c->T[j - 1][v][b];
    int r = pick(t, ww, Mx * My);
    tb_chain(t, x, y, r / My, r % My);
    return;
  }
  if (q == 1) {
    const R(*Qin)[NS] = c->QB[tri(c, x, y)];
    R ww[NS * NS];
    for (int a2 = 0; a2 < Mx; a2++)
      for (int b2 = 0; b2 < My; b2++)
        ww[a2 * My + b2] =
            c->T[i][a][a2] * Qin[a2][b2] * c->T[j - 1][b2][b] * stackf(c, i, a, j, b, a2, b2);
    int r = pick(t, ww, Mx * My);
    tb_qb(t, x, y, r / My, r % My);
    return;
  }
  if (q < 2 + 2 * MAXLOOP) {
    int L = (q - 2) / 2 + 1;
    if ((q - 2) % 2 == 0) {
      int l = j - 1 - L;
      const R(*Q)[NS] = c->QB[tri(c, x, l)];
      const R(*Cr)[NS] = c->C[tri(c, l, j)];
      R ww[NS * NS];
      int Ml = c->M[l];
      for (int a2 = 0; a2 < Mx; a2++)
        for (int e = 0; e < Ml; e++) ww[a2 * Ml + e] = c->T[i][a][a2] * Q[a2][e] * Cr[e][b];
      int r = pick(t, ww, Mx * Ml);
      tb_qb(t, x, l, r / Ml, r % Ml);
      tb_chain(t, l, j, r % Ml, b);
    } else {
      int k = i + 1 + L;
      const R(*Q)[NS] = c->QB[tri(c, k, y)];
      const R(*Cl)[NS] = c->C[tri(c, i, k)];
      R ww[NS * NS];
      int Mk = c->M[k];
      for (int e = 0; e < Mk; e++)
        for (int b2 = 0; b2 < My; b2++) ww[e * My + b2] = Cl[a][e] * Q[e][b2] * c->T[j - 1][b2][b];
      int r = pick(t, ww, Mk * My);
      tb_chain(t, i, k, a, r / My);
      tb_qb(t, k, y, r / My, r % My);
    }
    return;
  }
  if (q == nalt - 1) {
    const R(*Q2)[NPT] = c->QM2[tri(c, x, y)];
    int px[NPT], py[NPT];
    int nx = ports_of(c, x, px), ny = ports_of(c, y, py);
    R ww[NPT * NPT];
    for (int pi = 0; pi < nx; pi++)
      for (int qi = 0; qi < ny; qi++)
        ww[pi * ny + qi] = c->X[i][a + 6][px[pi]] * Q2[px[pi]][py[qi]] * c->X[j - 1][py[qi]][b + 6];
    int r = pick(t, ww, nx * ny);
    int p1 = px[r / ny], p2 = py[r % ny];
    tb_qm2(t, x, y, p1, p2);
    return;
  }
  /* interior loop: find (l1,l2) */
  idx = 2 + 2 * MAXLOOP;
  for (int l1 = 1; l1 <= MAXLOOP; l1++)
    for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++, idx++) {
      if (idx != q) continue;
      int k = i + 1 + l1, l = j - 1 - l2;
      const R(*C1)[NS] = c->C[tri(c, x, k - 1)];
      const R(*C2)[NS] = c->C[tri(c, l + 1, y)];
      const R(*Q)[NS] = c->QB[tri(c, k, l)];
      int Mw = c->M[k - 1], Mz = c->M[l + 1], Mk = c->M[k], Ml = c->M[l];
      /* states (u at x, w at k-1, z at l+1, v at y), then (k', l') */
      int tot = Mx * Mw * Mz * My;
      R *ww = malloc(sizeof(R) * tot);
      const R(*XI)[NS] = c->XI[tri(c, k, l)];
      int r = 0;
      for (int u = 0; u < Mx; u++)
        for (int w2 = 0; w2 < Mw; w2++)
          for (int z = 0; z < Mz; z++)
            for (int v = 0; v < My; v++)
              ww[r++] = c->T[i][a][u] * tmo(c, x, u, y, v) * c->T[j - 1][v][b] * C1[u][w2] *
                        XI[w2][z] * C2[z][v];
      int sel = pick(t, ww, tot);
      free(ww);
      int v = sel % My;
      sel /= My;
      int z = sel % Mz;
      sel /= Mz;
      int w2 = sel % Mw;
      int u = sel / Mw;
      R w3[NS * NS];
      for (int kk = 0; kk < Mk; kk++)
        for (int ll = 0; ll < Ml; ll++)
          w3[kk * Ml + ll] = c->T[k - 1][w2][kk] * Q[kk][ll] * c->T[l][ll][z];
      int r2 = pick(t, w3, Mk * Ml);
      tb_chain(t, x, k - 1, u, w2);
      set_state(t, k, r2 / Ml);
      set_state(t, l, r2 % Ml);
      if (c->T[k - 1][w2][r2 / Ml] == 0 || c->T[l][r2 % Ml][z] == 0) t->err = 4;
      tb_qb(t, k, l, r2 / Ml, r2 % Ml);
      tb_chain(t, l + 1, y, z, v);
      return;
    }
}

static void tb_ext(strace *t, int j, int a0, int port) {
  octx *c = t->c;
  while (1) {
    if (j == 0) {
      if (port != a0) t->err = 5;
      set_state(t, 0, a0);
      return;
    }
    int pq[NPT];
    int nq = ports_of(c, j - 1, pq);
    if (port < 6) {
      /* j unpaired */
      set_state(t, j, port);
      R w[NPT];
      for (int qi = 0; qi < nq; qi++) w[qi] = c->Q5[j - 1][a0][pq[qi]] * c->X[j - 1][pq[qi]][port];
      int r = pick(t, w, nq);
      j = j - 1;
      port = pq[r];
      continue;
    }
    int b = port - 6;
    /* j paired with k: k = 0 first, then k = 1..j-4 with (q, s) */
    int cnt = 1;
    for (int k = 1; k <= j - 4; k++) cnt += 2 * c->M[k - 1] * c->M[k];
    R *w = malloc(sizeof(R) * cnt);
    int idx = 0;
    w[idx++] = c->QB[tri(c, 0, j)][a0][b];
    for (int k = 1; k <= j - 4; k++) {
      int pk[NPT];
      int nk = ports_of(c, k - 1, pk);
      const R(*Qb)[NS] = c->QB[tri(c, k, j)];
      for (int qi = 0; qi < nk; qi++)
        for (int s = 0; s < c->M[k]; s++)
          w[idx++] = c->Q5[k - 1][a0][pk[qi]] * c->X[k - 1][pk[qi]][s + 6] * Qb[s][b];
    }
    int q = pick(t, w, cnt);
    free(w);
    if (q == 0) {
      tb_qb(t, 0, j, a0, b);
      return;
    }
    idx = 1;
    for (int k = 1; k <= j - 4; k++) {
      int pk[NPT];
      int nk = ports_of(c, k - 1, pk);
      int span = nk * c->M[k];
      if (q < idx + span) {
        int r = q - idx;
        int qp = pk[r / c->M[k]], s = r % c->M[k];
        tb_qb(t, k, j, s, b);
        j = k - 1;
        port = qp;
        break;
      }
      idx += span;
    }
  }
}

/* codons[ns*m] = sense codon id per residue; partner[ns*n] = partner or -1. */
int or_sample(const double *params, const int *res, int m, const double *lw, const double *pb,
              int nsamples, uint64_t seed, int *codons, int *partner) {
  if (m < 1 || nsamples < 0) return OR_EINVAL;
  octx c;
  int rc = setup(&c, params, res, m, lw, pb, NULL, 0);
  if (rc) {
    free_ctx(&c);
    return rc == -1 ? OR_EINVAL : OR_ENOMEM;
  }
  inside(&c);
  int n = c.n;
  int *st = malloc(sizeof(int) * n);
  int err = 0;
  for (int smp = 0; smp < nsamples; smp++) {
    strace t;
    t.c = &c;
    t.g.s = seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(smp + 1);
    t.state = st;
    t.partner = partner + (size_t)smp * n;
    t.err = 0;
    for (int p = 0; p < n; p++) {
      st[p] = -1;
      t.partner[p] = -1;
    }
    /* top: (a0, port at n-1) */
    int pp[NPT];
    int np = ports_of(&c, n - 1, pp);
    R w[NS * NPT];
    for (int a = 0; a < c.M[0]; a++)
      for (int qi = 0; qi < np; qi++) w[a * np + qi] = c.u0[a] * c.Q5[n - 1][a][pp[qi]];
    int r = pick(&t, w, c.M[0] * np);
    tb_ext(&t, n - 1, r / np, pp[r % np]);
    for (int rr = 0; rr < m; rr++) {
      int p = 3 * rr;
      if (st[p] < 0 || st[p + 1] != st[p] || st[p + 2] != st[p]) t.err = 6;
      codons[(size_t)smp * m + rr] = st[p] >= 0 ? c.cid[p][st[p]] : -1;
    }
    if (t.err) err = t.err;
  }
  free(st);
  free_ctx(&c);
  return err ? 100 + err : OR_OK;
}

/* Sense codon id list of amino acid index aa (codon-id order); returns count. */
int or_codons_of(int aa, int *out) {
  if (aa < 0 || aa >= 20) return 0;
  int cnt = 0;
  for (int k = 0; k < 64; k++)
    if (OR_CODE64[k] == OR_AA[aa]) out[cnt++] = sense_id(k);
  return cnt;
}

/* ================================================================ MFE
 * Minimum free energy over (codon sequence, structure): paper Section
 * "Minimization" (Eq. min-problem) -- the zero-temperature limit obtained by
 * replacing the sum-product semiring of the partition function with the
 * min-sum (tropical) semiring (SI "Generalization via evaluation algebras").
 * The recursions are those of the inside pass above, statement for
 * statement, with every sum a minimum and every product a sum of costs.
 *
 * Costs are exact integers: every elementary energy term (stack, hairpin,
 * bulge, interior, mismatch, dangle, a, b, c, and each codon log-weight and
 * codon-pair bonus converted to kcal/mol as -kT w) is rounded to the nearest
 * multiple of 2^-32 kcal/mol (round half away from zero) once, and all
 * recursions add these integers.  The minimum is then exact and independent
 * of the order of evaluation, so any implementation of the same model gives
 * the identical value.  kT = 1.98717e-3 (T + 273.15) and -kT w are evaluated
 * in binary64; the hairpin extrapolation H(30) + 1.07856 ln(L/30) too.
 * ================================================================ */

typedef long long Q;
#define QINF (1LL << 60)

static Q qcost(double e) { return llround(e * 4294967296.0); }
static Q qadd(Q a, Q b) { return (a >= QINF || b >= QINF) ? QINF : a + b; }
static Q qmin(Q a, Q b) { return a < b ? a : b; }

typedef struct {
  int n, m;
  int *M;
  int (*base)[NS];
  int (*cid)[NS];
  Q st[6][6], Hl[MAXLOOP + 1], Bu[MAXLOOP + 1], In[MAXLOOP + 1];
  Q tm[4][4], d5[4][4], d3[4][4], ca, cb, cc;
  double H30, kT;
  Q (*T)[NS][NS];   /* transfer cost p -> p+1 */
  Q (*X)[NPT][NPT]; /* typed transition cost */
  Q u0[NS];
  /* tables, triangular index as tri() */
  Q (*C)[NS][NS];
  Q (*QB)[NS][NS];
  Q (*XI)[NS][NS];
  Q (*QM1)[NS][NPT];
  Q (*QM)[NPT][NPT];
  Q (*QM2)[NPT][NPT];
  Q (*Q5)[NS][NPT];
  Q mfe;
} mctx;

/* ports of a position with M codon states: states a (type U) then a + 6 (type P) */
static int ports_of_m(int M, int *out) {
  int k = 0;
  for (int t = 0; t < 2; t++)
    for (int a = 0; a < M; a++) out[k++] = a + 6 * t;
  return k;
}

static inline size_t mtri(const mctx *c, int i, int j) {
  return (size_t)i * c->n - (size_t)i * (i - 1) / 2 + (size_t)(j - i);
}

static Q m_hairpin(const mctx *c, int L) {
  if (L <= MAXLOOP) return c->Hl[L];
  return qcost(c->H30 + 1.07856 * log((double)L / MAXLOOP));
}

static void m_free(mctx *c) {
  free(c->M); free(c->base); free(c->cid); free(c->T); free(c->X);
  free(c->C); free(c->QB); free(c->XI); free(c->QM1); free(c->QM); free(c->QM2); free(c->Q5);
  memset(c, 0, sizeof(*c));
}

static void qfill(Q *p, size_t cnt) {
  for (size_t k = 0; k < cnt; k++) p[k] = QINF;
}

static int m_setup(mctx *c, const double *params, const int *res, int m, const double *lw, const double *pb) {
  memset(c, 0, sizeof(*c));
  c->m = m;
  c->n = 3 * m;
  int n = c->n;
  c->kT = 1.98717e-3 * (params[180] + 273.15);
  for (int x = 0; x < 6; x++)
    for (int y = 0; y < 6; y++) c->st[x][y] = qcost(params[6 * x + y]);
  for (int L = 0; L <= MAXLOOP; L++) {
    c->Hl[L] = qcost(params[36 + L]);
    c->Bu[L] = qcost(params[67 + L]);
    c->In[L] = qcost(params[98 + L]);
  }
  c->H30 = params[36 + MAXLOOP];
  for (int x = 0; x < 4; x++)
    for (int y = 0; y < 4; y++) {
      c->tm[x][y] = qcost(params[129 + 4 * x + y]);
      c->d5[x][y] = qcost(params[145 + 4 * x + y]);
      c->d3[x][y] = qcost(params[161 + 4 * x + y]);
    }
  c->ca = qcost(params[177]);
  c->cb = qcost(params[178]);
  c->cc = qcost(params[179]);
  c->M = calloc(n, sizeof(int));
  c->base = calloc(n, sizeof(*c->base));
  c->cid = calloc(n, sizeof(*c->cid));
  c->T = malloc(n * sizeof(*c->T));
  c->X = malloc(n * sizeof(*c->X));
  if (!c->M || !c->base || !c->cid || !c->T || !c->X) return -2;
  for (int r = 0; r < m; r++) {
    if (res[r] < 0 || res[r] >= 20) return -1;
    char aa = OR_AA[res[r]];
    int cnt = 0, cods[NS];
    for (int k = 0; k < 64; k++)
      if (OR_CODE64[k] == aa) cods[cnt++] = k;
    for (int off = 0; off < 3; off++) {
      int p = 3 * r + off;
      c->M[p] = cnt;
      for (int a = 0; a < cnt; a++) {
        c->base[p][a] = codon_base(cods[a], off);
        c->cid[p][a] = sense_id(cods[a]);
      }
    }
  }
  qfill(&c->T[0][0][0], (size_t)n * NS * NS);
  qfill(&c->X[0][0][0], (size_t)n * NPT * NPT);
  for (int p = 0; p + 1 < n; p++) {
    int r1 = (p + 1) / 3;
    for (int a = 0; a < c->M[p]; a++)
      for (int b = 0; b < c->M[p + 1]; b++) {
        Q t;
        if (p % 3 != 2) {
          t = (a == b) ? 0 : QINF;
        } else {
          t = qcost(-(c->kT * (lw ? lw[6 * r1 + b] : 0.0)));
          t += qcost(-(c->kT * (pb ? pb[61 * c->cid[p][a] + c->cid[p + 1][b]] : 0.0)));
        }
        c->T[p][a][b] = t;
        int x = c->base[p][a], y = c->base[p + 1][b];
        for (int t1 = 0; t1 < 2; t1++)
          for (int t2 = 0; t2 < 2; t2++) {
            Q f = t;
            if (t1 == TP) f = qadd(f, c->d3[x][y]);
            if (t2 == TP) f = qadd(f, c->d5[y][x]);
            c->X[p][a + 6 * t1][b + 6 * t2] = f;
          }
      }
  }
  for (int a = 0; a < NS; a++) c->u0[a] = a < c->M[0] ? qcost(-(c->kT * (lw ? lw[a] : 0.0))) : QINF;
  size_t ncell = (size_t)n * (n + 1) / 2;
  c->C = malloc(ncell * sizeof(*c->C));
  c->QB = malloc(ncell * sizeof(*c->QB));
  c->XI = malloc(ncell * sizeof(*c->XI));
  c->QM1 = malloc(ncell * sizeof(*c->QM1));
  c->QM = malloc(ncell * sizeof(*c->QM));
  c->QM2 = malloc(ncell * sizeof(*c->QM2));
  c->Q5 = malloc(n * sizeof(*c->Q5));
  if (!c->C || !c->QB || !c->XI || !c->QM1 || !c->QM || !c->QM2 || !c->Q5) return -2;
  qfill(&c->C[0][0][0], ncell * NS * NS);
  qfill(&c->QB[0][0][0], ncell * NS * NS);
  qfill(&c->XI[0][0][0], ncell * NS * NS);
  qfill(&c->QM1[0][0][0], ncell * NS * NPT);
  qfill(&c->QM[0][0][0], ncell * NPT * NPT);
  qfill(&c->QM2[0][0][0], ncell * NPT * NPT);
  qfill(&c->Q5[0][0][0], (size_t)n * NS * NPT);
  return 0;
}

static int m_pairable(const mctx *c, int i, int a, int j, int b) {
  return j - i >= 4 && pair_type(c->base[i][a], c->base[j][b]) >= 0;
}
static Q m_tmo(const mctx *c, int x, int u, int y, int v) { return c->tm[c->base[x][u]][c->base[y][v]]; }
static Q m_tmi(const mctx *c, int k, int w, int l, int z) { return c->tm[c->base[l + 1][z]][c->base[k - 1][w]]; }

static void m_chain(mctx *c, int i, int j) {
  Q(*Cij)[NS] = c->C[mtri(c, i, j)];
  if (i == j) {
    for (int a = 0; a < c->M[i]; a++) Cij[a][a] = 0;
    return;
  }
  const Q(*Cn)[NS] = c->C[mtri(c, i + 1, j)];
  for (int a = 0; a < c->M[i]; a++)
    for (int s = 0; s < c->M[i + 1]; s++)
      for (int b = 0; b < c->M[j]; b++) Cij[a][b] = qmin(Cij[a][b], qadd(c->T[i][a][s], Cn[s][b]));
}

/* hairpin + interior loops of the loop closed by (i,j), before the outer
 * mismatch and transfers: M_{i+1} x M_{j-1} (inner_sum of the inside pass) */
static void m_inner(const mctx *c, int i, int j, Q S[NS][NS]) {
  int x = i + 1, y = j - 1;
  Q h = m_hairpin(c, j - i - 1);
  const Q(*Ch)[NS] = c->C[mtri(c, x, y)];
  for (int u = 0; u < NS; u++)
    for (int v = 0; v < NS; v++) S[u][v] = QINF;
  for (int u = 0; u < c->M[x]; u++)
    for (int v = 0; v < c->M[y]; v++) S[u][v] = qadd(h, Ch[u][v]);
  for (int l1 = 1; l1 <= MAXLOOP; l1++)
    for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++) {
      int k = i + 1 + l1, l = j - 1 - l2;
      if (l - k < 4) continue;
      Q w = c->In[l1 + l2];
      const Q(*C1)[NS] = c->C[mtri(c, x, k - 1)];
      const Q(*XI)[NS] = c->XI[mtri(c, k, l)];
      const Q(*C2)[NS] = c->C[mtri(c, l + 1, y)];
      for (int u = 0; u < c->M[x]; u++)
        for (int w2 = 0; w2 < c->M[k - 1]; w2++)
          for (int z = 0; z < c->M[l + 1]; z++)
            for (int v = 0; v < c->M[y]; v++)
              S[u][v] = qmin(S[u][v], qadd(qadd(w, C1[u][w2]), qadd(XI[w2][z], C2[z][v])));
    }
}

static Q m_stack(const mctx *c, int i, int a, int j, int b, int a2, int b2) {
  int o = pair_type(c->base[i][a], c->base[j][b]);
  int in = pair_type(c->base[i + 1][a2], c->base[j - 1][b2]);
  if (o < 0 || in < 0) return QINF;
  return c->st[o][in];
}

static void m_qb(mctx *c, int i, int j) {
  Q acc[NS][NS];
  int Mi = c->M[i], Mj = c->M[j], Mx = c->M[i + 1], My = c->M[j - 1];
  for (int a = 0; a < NS; a++)
    for (int b = 0; b < NS; b++) acc[a][b] = QINF;
  Q S[NS][NS];
  m_inner(c, i, j, S);
  for (int a = 0; a < Mi; a++)
    for (int b = 0; b < Mj; b++)
      for (int u = 0; u < Mx; u++)
        for (int v = 0; v < My; v++) {
          Q k = qadd(S[u][v], m_tmo(c, i + 1, u, j - 1, v));
          acc[a][b] = qmin(acc[a][b], qadd(qadd(c->T[i][a][u], k), c->T[j - 1][v][b]));
        }
  if (j - i - 2 >= 4) { /* stack */
    const Q(*Qin)[NS] = c->QB[mtri(c, i + 1, j - 1)];
    for (int a = 0; a < Mi; a++)
      for (int b = 0; b < Mj; b++)
        for (int a2 = 0; a2 < Mx; a2++)
          for (int b2 = 0; b2 < My; b2++)
            acc[a][b] = qmin(acc[a][b], qadd(qadd(c->T[i][a][a2], Qin[a2][b2]),
                                             qadd(c->T[j - 1][b2][b], m_stack(c, i, a, j, b, a2, b2))));
  }
  for (int L = 1; L <= MAXLOOP; L++) {
    int l = j - 1 - L; /* 3' bulge: inner pair (i+1, l) */
    if (l - (i + 1) >= 4) {
      const Q(*Qi)[NS] = c->QB[mtri(c, i + 1, l)];
      const Q(*Cr)[NS] = c->C[mtri(c, l, j)];
      for (int a = 0; a < Mi; a++)
        for (int a2 = 0; a2 < Mx; a2++)
          for (int s = 0; s < c->M[l]; s++)
            for (int b = 0; b < Mj; b++)
              acc[a][b] = qmin(acc[a][b], qadd(qadd(c->Bu[L], c->T[i][a][a2]), qadd(Qi[a2][s], Cr[s][b])));
    }
    int k = i + 1 + L; /* 5' bulge: inner pair (k, j-1) */
    if ((j - 1) - k >= 4) {
      const Q(*Qi)[NS] = c->QB[mtri(c, k, j - 1)];
      const Q(*Cl)[NS] = c->C[mtri(c, i, k)];
      for (int a = 0; a < Mi; a++)
        for (int s = 0; s < c->M[k]; s++)
          for (int b2 = 0; b2 < My; b2++)
            for (int b = 0; b < Mj; b++)
              acc[a][b] = qmin(acc[a][b], qadd(qadd(c->Bu[L], Cl[a][s]), qadd(Qi[s][b2], c->T[j - 1][b2][b])));
    }
  }
  if (j - i - 2 >= 9) { /* multiloop closed by (i,j) */
    const Q(*Q2)[NPT] = c->QM2[mtri(c, i + 1, j - 1)];
    int px[NPT], py[NPT];
    int nx = ports_of_m(c->M[i + 1], px), ny = ports_of_m(c->M[j - 1], py);
    Q w = qadd(c->ca, c->cc);
    for (int a = 0; a < Mi; a++)
      for (int b = 0; b < Mj; b++)
        for (int pi = 0; pi < nx; pi++)
          for (int qi = 0; qi < ny; qi++)
            acc[a][b] = qmin(acc[a][b], qadd(qadd(w, c->X[i][a + 6][px[pi]]),
                                             qadd(Q2[px[pi]][py[qi]], c->X[j - 1][py[qi]][b + 6])));
  }
  Q(*QBij)[NS] = c->QB[mtri(c, i, j)];
  for (int a = 0; a < Mi; a++)
    for (int b = 0; b < Mj; b++) QBij[a][b] = m_pairable(c, i, a, j, b) ? acc[a][b] : QINF;
}

static void m_xi(mctx *c, int k, int l) {
  if (k < 1 || l > c->n - 2) return;
  const Q(*Qk)[NS] = c->QB[mtri(c, k, l)];
  Q(*XI)[NS] = c->XI[mtri(c, k, l)];
  for (int w = 0; w < c->M[k - 1]; w++)
    for (int z = 0; z < c->M[l + 1]; z++) {
      Q s = QINF;
      for (int a = 0; a < c->M[k]; a++)
        for (int b = 0; b < c->M[l]; b++) s = qmin(s, qadd(qadd(c->T[k - 1][w][a], Qk[a][b]), c->T[l][b][z]));
      XI[w][z] = qadd(s, m_tmi(c, k, w, l, z));
    }
}

static void m_qm1(mctx *c, int i, int j) {
  Q(*Q1)[NPT] = c->QM1[mtri(c, i, j)];
  const Q(*QBij)[NS] = c->QB[mtri(c, i, j)];
  for (int a = 0; a < c->M[i]; a++)
    for (int b = 0; b < c->M[j]; b++) Q1[a][b + 6] = qadd(c->cc, QBij[a][b]);
  for (int l = i + 4; l <= j - 1; l++) {
    const Q(*Qil)[NS] = c->QB[mtri(c, i, l)];
    const Q(*Cr)[NS] = c->C[mtri(c, l + 1, j)];
    Q w = c->cc + (Q)(j - l) * c->cb;
    for (int a = 0; a < c->M[i]; a++)
      for (int s = 0; s < c->M[l]; s++)
        for (int e = 0; e < c->M[l + 1]; e++)
          for (int b = 0; b < c->M[j]; b++)
            Q1[a][b] = qmin(Q1[a][b], qadd(qadd(w, Qil[a][s]), qadd(c->X[l][s + 6][e], Cr[e][b])));
  }
}

static void m_qm(mctx *c, int i, int j) {
  Q(*QM)[NPT] = c->QM[mtri(c, i, j)];
  const Q(*Q1)[NPT] = c->QM1[mtri(c, i, j)];
  int pi_[NPT], pj[NPT];
  int ni = ports_of_m(c->M[i], pi_), nj = ports_of_m(c->M[j], pj);
  for (int a = 0; a < c->M[i]; a++)
    for (int qi = 0; qi < nj; qi++) QM[a + 6][pj[qi]] = qmin(QM[a + 6][pj[qi]], Q1[a][pj[qi]]);
  for (int k = i + 1; k <= j - 4; k++) {
    const Q(*Qp)[NPT] = c->QM[mtri(c, i, k - 1)];
    const Q(*Cu)[NS] = c->C[mtri(c, i, k - 1)];
    const Q(*Qk)[NPT] = c->QM1[mtri(c, k, j)];
    int pq[NPT];
    int nq = ports_of_m(c->M[k - 1], pq);
    Q un = (Q)(k - i) * c->cb;
    for (int ri = 0; ri < ni; ri++) {
      int p = pi_[ri];
      for (int qi = 0; qi < nq; qi++) {
        int q = pq[qi];
        Q left = Qp[p][q]; /* >= 1 branch in [i, k-1] */
        if (p < 6 && q < 6) left = qmin(left, qadd(un, Cu[p][q])); /* [i, k-1] unpaired */
        for (int b = 0; b < c->M[k]; b++) {
          Q t = qadd(left, c->X[k - 1][q][b + 6]);
          for (int si = 0; si < nj; si++) QM[p][pj[si]] = qmin(QM[p][pj[si]], qadd(t, Qk[b][pj[si]]));
        }
      }
    }
  }
}

static void m_qm2(mctx *c, int i, int j) {
  Q(*Q2)[NPT] = c->QM2[mtri(c, i, j)];
  int pi_[NPT], pj[NPT];
  int ni = ports_of_m(c->M[i], pi_), nj = ports_of_m(c->M[j], pj);
  for (int k = i + 5; k <= j - 4; k++) {
    const Q(*Qp)[NPT] = c->QM[mtri(c, i, k - 1)];
    const Q(*Qk)[NPT] = c->QM1[mtri(c, k, j)];
    int pq[NPT];
    int nq = ports_of_m(c->M[k - 1], pq);
    for (int ri = 0; ri < ni; ri++)
      for (int qi = 0; qi < nq; qi++)
        for (int b = 0; b < c->M[k]; b++) {
          Q t = qadd(Qp[pi_[ri]][pq[qi]], c->X[k - 1][pq[qi]][b + 6]);
          for (int si = 0; si < nj; si++) Q2[pi_[ri]][pj[si]] = qmin(Q2[pi_[ri]][pj[si]], qadd(t, Qk[b][pj[si]]));
        }
  }
}

static void m_exterior(mctx *c) {
  int n = c->n;
  for (int a = 0; a < c->M[0]; a++) c->Q5[0][a][a] = 0;
  for (int j = 1; j < n; j++) {
    Q(*Q5j)[NPT] = c->Q5[j];
    int pp[NPT];
    int np = ports_of_m(c->M[j - 1], pp);
    for (int a = 0; a < c->M[0]; a++)
      for (int b = 0; b < c->M[j]; b++)
        for (int qi = 0; qi < np; qi++)
          Q5j[a][b] = qmin(Q5j[a][b], qadd(c->Q5[j - 1][a][pp[qi]], c->X[j - 1][pp[qi]][b]));
    const Q(*QB0)[NS] = c->QB[mtri(c, 0, j)];
    for (int a = 0; a < c->M[0]; a++)
      for (int b = 0; b < c->M[j]; b++) Q5j[a][b + 6] = qmin(Q5j[a][b + 6], QB0[a][b]);
    for (int k = 1; k <= j - 4; k++) {
      int pq[NPT];
      int nq = ports_of_m(c->M[k - 1], pq);
      const Q(*QBk)[NS] = c->QB[mtri(c, k, j)];
      for (int a = 0; a < c->M[0]; a++)
        for (int qi = 0; qi < nq; qi++)
          for (int s = 0; s < c->M[k]; s++) {
            Q t = qadd(c->Q5[k - 1][a][pq[qi]], c->X[k - 1][pq[qi]][s + 6]);
            for (int b = 0; b < c->M[j]; b++) Q5j[a][b + 6] = qmin(Q5j[a][b + 6], qadd(t, QBk[s][b]));
          }
    }
  }
  Q best = QINF;
  int pp[NPT];
  int np = ports_of_m(c->M[n - 1], pp);
  for (int a = 0; a < c->M[0]; a++)
    for (int qi = 0; qi < np; qi++) best = qmin(best, qadd(c->u0[a], c->Q5[n - 1][a][pp[qi]]));
  c->mfe = best;
}

static void m_inside(mctx *c) {
  int n = c->n;
  for (int d = 0; d < n; d++) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n - d; i++) {
      int j = i + d;
      m_chain(c, i, j);
      if (d >= 4) {
        m_qb(c, i, j);
        m_xi(c, i, j);
        m_qm1(c, i, j);
        m_qm(c, i, j);
        if (d >= 9) m_qm2(c, i, j);
      }
    }
  }
  m_exterior(c);
}

/* ---------------------------------------------------------------- MFE traceback
 * Follows the recursions back from the minimum: at every table entry the
 * first alternative (in the order each routine states) whose cost equals the
 * entry is taken.  Costs are exact integers, so the equality test is exact.
 * Writes the codon state of every position and the pairing partner. */

typedef struct {
  mctx *c;
  int *state, *partner;
  int err;
} mtrace;

static void mt_state(mtrace *t, int p, int a) {
  if (t->state[p] >= 0 && t->state[p] != a) t->err = 2;
  t->state[p] = a;
}

static void mt_chain(mtrace *t, int x, int y, int a, int b) {
  mctx *c = t->c;
  mt_state(t, x, a);
  int cur = a;
  for (int p = x; p < y; p++) {
    Q want = c->C[mtri(c, p, y)][cur][b];
    int nxt = -1;
    for (int s = 0; s < c->M[p + 1] && nxt < 0; s++)
      if (qadd(c->T[p][cur][s], c->C[mtri(c, p + 1, y)][s][b]) == want) nxt = s;
    if (nxt < 0) {
      t->err = 3;
      return;
    }
    cur = nxt;
    mt_state(t, p + 1, cur);
  }
}

static void mt_qb(mtrace *t, int i, int j, int a, int b);
static void mt_qm(mtrace *t, int i, int j, int p1, int p2);

static void mt_qm1(mtrace *t, int i, int j, int a, int p2) {
  mctx *c = t->c;
  if (p2 >= 6) { /* the branch ends at j */
    mt_qb(t, i, j, a, p2 - 6);
    return;
  }
  Q want = c->QM1[mtri(c, i, j)][a][p2];
  /* branch (i, l) then j - l unpaired: l ascending, state s at l, e at l+1 */
  for (int l = i + 4; l <= j - 1; l++) {
    Q w = c->cc + (Q)(j - l) * c->cb;
    for (int s = 0; s < c->M[l]; s++)
      for (int e = 0; e < c->M[l + 1]; e++)
        if (qadd(qadd(w, c->QB[mtri(c, i, l)][a][s]), qadd(c->X[l][s + 6][e], c->C[mtri(c, l + 1, j)][e][p2])) ==
            want) {
          mt_qb(t, i, l, a, s);
          mt_chain(t, l + 1, j, e, p2);
          return;
        }
  }
  t->err = 4;
}

static void mt_qm2(mtrace *t, int i, int j, int p1, int p2) {
  mctx *c = t->c;
  Q want = c->QM2[mtri(c, i, j)][p1][p2];
  /* last branch starts at k (ascending), port q at k-1, state b at k */
  for (int k = i + 5; k <= j - 4; k++) {
    int pq[NPT];
    int nq = ports_of_m(c->M[k - 1], pq);
    for (int qi = 0; qi < nq; qi++)
      for (int b = 0; b < c->M[k]; b++)
        if (qadd(qadd(c->QM[mtri(c, i, k - 1)][p1][pq[qi]], c->X[k - 1][pq[qi]][b + 6]),
                 c->QM1[mtri(c, k, j)][b][p2]) == want) {
          mt_qm(t, i, k - 1, p1, pq[qi]);
          mt_qm1(t, k, j, b, p2);
          return;
        }
  }
  t->err = 5;
}

static void mt_qm(mtrace *t, int i, int j, int p1, int p2) {
  mctx *c = t->c;
  Q want = c->QM[mtri(c, i, j)][p1][p2];
  if (p1 >= 6 && c->QM1[mtri(c, i, j)][p1 - 6][p2] == want) { /* one branch starting at i */
    mt_qm1(t, i, j, p1 - 6, p2);
    return;
  }
  /* k ascending; port q at k-1; prefix [i, k-1] unpaired, then with >= 1 branch; state b at k */
  for (int k = i + 1; k <= j - 4; k++) {
    int pq[NPT];
    int nq = ports_of_m(c->M[k - 1], pq);
    Q un = (Q)(k - i) * c->cb;
    for (int qi = 0; qi < nq; qi++)
      for (int kind = 0; kind < 2; kind++) {
        Q left;
        if (kind == 0) left = (p1 < 6 && pq[qi] < 6) ? qadd(un, c->C[mtri(c, i, k - 1)][p1][pq[qi]]) : QINF;
        else left = c->QM[mtri(c, i, k - 1)][p1][pq[qi]];
        for (int b = 0; b < c->M[k]; b++)
          if (qadd(qadd(left, c->X[k - 1][pq[qi]][b + 6]), c->QM1[mtri(c, k, j)][b][p2]) == want) {
            if (kind == 0) mt_chain(t, i, k - 1, p1, pq[qi]);
            else mt_qm(t, i, k - 1, p1, pq[qi]);
            mt_qm1(t, k, j, b, p2);
            return;
          }
      }
  }
  t->err = 6;
}

static void mt_qb(mtrace *t, int i, int j, int a, int b) {
  mctx *c = t->c;
  int Mx = c->M[i + 1], My = c->M[j - 1];
  Q want = c->QB[mtri(c, i, j)][a][b];
  t->partner[i] = j;
  t->partner[j] = i;
  mt_state(t, i, a);
  mt_state(t, j, b);
  int x = i + 1, y = j - 1;
  /* 1. hairpin, then interior loops (l1, l2 as in m_inner), over (u, v) ascending */
  for (int u = 0; u < Mx; u++)
    for (int v = 0; v < My; v++) {
      Q outer = qadd(qadd(c->T[i][a][u], c->T[j - 1][v][b]), m_tmo(c, x, u, y, v));
      if (outer >= QINF) continue;
      if (qadd(outer, qadd(m_hairpin(c, j - i - 1), c->C[mtri(c, x, y)][u][v])) == want) {
        mt_chain(t, x, y, u, v);
        return;
      }
      for (int l1 = 1; l1 <= MAXLOOP; l1++)
        for (int l2 = 1; l1 + l2 <= MAXLOOP; l2++) {
          int k = i + 1 + l1, l = j - 1 - l2;
          if (l - k < 4) continue;
          for (int w2 = 0; w2 < c->M[k - 1]; w2++)
            for (int z = 0; z < c->M[l + 1]; z++) {
              Q v2 = qadd(qadd(c->In[l1 + l2], c->C[mtri(c, x, k - 1)][u][w2]),
                          qadd(c->XI[mtri(c, k, l)][w2][z], c->C[mtri(c, l + 1, y)][z][v]));
              if (qadd(outer, v2) != want) continue;
              /* the inner pair (k, l): states a2 at k, b2 at l */
              const Q xi = qadd(c->XI[mtri(c, k, l)][w2][z], 0);
              for (int a2 = 0; a2 < c->M[k]; a2++)
                for (int b2 = 0; b2 < c->M[l]; b2++)
                  if (qadd(qadd(c->T[k - 1][w2][a2], c->QB[mtri(c, k, l)][a2][b2]),
                           qadd(c->T[l][b2][z], m_tmi(c, k, w2, l, z))) == xi) {
                    mt_chain(t, x, k - 1, u, w2);
                    mt_chain(t, l + 1, y, z, v);
                    mt_qb(t, k, l, a2, b2);
                    return;
                  }
              t->err = 7;
              return;
            }
        }
    }
  /* 2. stack: states (a2, b2) ascending */
  if (j - i - 2 >= 4)
    for (int a2 = 0; a2 < Mx; a2++)
      for (int b2 = 0; b2 < My; b2++)
        if (qadd(qadd(c->T[i][a][a2], c->QB[mtri(c, i + 1, j - 1)][a2][b2]),
                 qadd(c->T[j - 1][b2][b], m_stack(c, i, a, j, b, a2, b2))) == want) {
          mt_qb(t, i + 1, j - 1, a2, b2);
          return;
        }
  /* 3. bulges: L ascending, the 3' bulge before the 5' bulge */
  for (int L = 1; L <= MAXLOOP; L++) {
    int l = j - 1 - L;
    if (l - (i + 1) >= 4)
      for (int a2 = 0; a2 < Mx; a2++)
        for (int s = 0; s < c->M[l]; s++)
          if (qadd(qadd(c->Bu[L], c->T[i][a][a2]), qadd(c->QB[mtri(c, i + 1, l)][a2][s], c->C[mtri(c, l, j)][s][b])) ==
              want) {
            mt_qb(t, i + 1, l, a2, s);
            mt_chain(t, l, j, s, b);
            return;
          }
    int k = i + 1 + L;
    if ((j - 1) - k >= 4)
      for (int s = 0; s < c->M[k]; s++)
        for (int b2 = 0; b2 < My; b2++)
          if (qadd(qadd(c->Bu[L], c->C[mtri(c, i, k)][a][s]), qadd(c->QB[mtri(c, k, j - 1)][s][b2], c->T[j - 1][b2][b])) ==
              want) {
            mt_chain(t, i, k, a, s);
            mt_qb(t, k, j - 1, s, b2);
            return;
          }
  }
  /* 4. multiloop: ports at i+1 and j-1 in port order */
  if (j - i - 2 >= 9) {
    int px[NPT], py[NPT];
    int nx = ports_of_m(Mx, px), ny = ports_of_m(My, py);
    Q w = qadd(c->ca, c->cc);
    for (int pi = 0; pi < nx; pi++)
      for (int qi = 0; qi < ny; qi++)
        if (qadd(qadd(w, c->X[i][a + 6][px[pi]]),
                 qadd(c->QM2[mtri(c, x, y)][px[pi]][py[qi]], c->X[j - 1][py[qi]][b + 6])) == want) {
          mt_state(t, x, px[pi] % 6);
          mt_state(t, y, py[qi] % 6);
          mt_qm2(t, x, y, px[pi], py[qi]);
          return;
        }
  }
  t->err = 8;
}

static void mt_ext(mtrace *t, int j, int a0, int port) {
  mctx *c = t->c;
  if (j == 0) {
    mt_state(t, 0, a0);
    if (port != a0) t->err = 9;
    return;
  }
  Q want = c->Q5[j][a0][port];
  int pp[NPT];
  int np = ports_of_m(c->M[j - 1], pp);
  if (port < 6) { /* j unpaired: port at j-1 in port order */
    for (int qi = 0; qi < np; qi++)
      if (qadd(c->Q5[j - 1][a0][pp[qi]], c->X[j - 1][pp[qi]][port]) == want) {
        mt_state(t, j, port);
        mt_ext(t, j - 1, a0, pp[qi]);
        return;
      }
    t->err = 10;
    return;
  }
  int b = port - 6;
  if (c->QB[mtri(c, 0, j)][a0][b] == want) { /* a branch (0, j) */
    mt_qb(t, 0, j, a0, b);
    return;
  }
  for (int k = 1; k <= j - 4; k++) { /* last branch (k, j): k ascending, port at k-1, state at k */
    int pq[NPT];
    int nq = ports_of_m(c->M[k - 1], pq);
    for (int qi = 0; qi < nq; qi++)
      for (int s = 0; s < c->M[k]; s++)
        if (qadd(qadd(c->Q5[k - 1][a0][pq[qi]], c->X[k - 1][pq[qi]][s + 6]), c->QB[mtri(c, k, j)][s][b]) == want) {
          mt_qb(t, k, j, s, b);
          mt_ext(t, k - 1, a0, pq[qi]);
          return;
        }
  }
  t->err = 11;
}

/* MFE of (codon sequence, structure): *mfe_q = the minimum in units of 2^-32
 * kcal/mol (QINF if no configuration exists), *mfe_kcal the same in kcal/mol;
 * codons[m] (sense codon ids) and partner[n] (-1 unpaired) of one minimiser,
 * either may be NULL.  Returns 0, OR_EINVAL, OR_ENOMEM, or 100 + a traceback
 * inconsistency code. */
int or_mfe(const double *params, const int *res, int m, const double *lw, const double *pb, long long *mfe_q,
           double *mfe_kcal, int *codons, int *partner) {
  if (m < 1) return OR_EINVAL;
  mctx c;
  int rc = m_setup(&c, params, res, m, lw, pb);
  if (rc) {
    m_free(&c);
    return rc == -1 ? OR_EINVAL : OR_ENOMEM;
  }
  m_inside(&c);
  *mfe_q = c.mfe;
  *mfe_kcal = (double)c.mfe / 4294967296.0;
  int err = 0;
  if (codons || partner) {
    int n = c.n;
    int *state = malloc(n * sizeof(int)), *pt = malloc(n * sizeof(int));
    for (int p = 0; p < n; p++) state[p] = pt[p] = -1;
    mtrace t = {&c, state, pt, 0};
    int done = 0;
    int pp[NPT];
    int np = ports_of_m(c.M[n - 1], pp);
    for (int a = 0; a < c.M[0] && !done; a++)
      for (int qi = 0; qi < np && !done; qi++)
        if (qadd(c.u0[a], c.Q5[n - 1][a][pp[qi]]) == c.mfe) {
          mt_ext(&t, n - 1, a, pp[qi]);
          done = 1;
        }
    if (!done) t.err = 12;
    for (int p = 0; p < n && !t.err; p++)
      if (state[p] < 0) t.err = 13;
    if (codons)
      for (int r = 0; r < m; r++) codons[r] = t.err ? -1 : c.cid[3 * r][state[3 * r]];
    if (partner)
      for (int p = 0; p < n; p++) partner[p] = pt[p];
    err = t.err;
    free(state);
    free(pt);
  }
  m_free(&c);
  return err ? 100 + err : OR_OK;
}
