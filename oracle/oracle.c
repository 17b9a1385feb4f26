/*
 * CPU FP64 oracle for the batched element-local contraction and for the MLP
 * cost model.  TEST INFRASTRUCTURE ONLY: it is called by the test suite, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the library.
 * It shares no code, header or constant with the CUDA path.
 *
 * Everything here is the plain definition written out, in float64, with no
 * blocking, fusion or reordering of any sum:
 *
 *   contraction  out[f,e,i] = sum_j D[f,i,j] * u[e,j]
 *     This is the untransformed loop nest of the dG FEM volume workload
 *     (Table 1), stated in the paper's data model as a loop domain
 *     { [f,e,i,j] : 0<=f<F and 0<=e<E and 0<=i,j<N } plus one instruction with a
 *     sum reduction over j (Section 2.1).  Every transformation of Section 2.4
 *     (split_iname of Eq. 1, unrolling, ilp/vec tags, layout tags, prefetch)
 *     claims to reproduce exactly this result, and the unordered semantics of
 *     Section 2.3 make the traversal order irrelevant, so j runs ascending and
 *     the loop over elements may run in parallel.
 *
 *   bf16 rounding   round-to-nearest, ties-to-even, of a binary32 value to its
 *     upper 16 bits (IEEE 754 rounding applied to the bfloat16 format).
 *   bf16 split      x = hi + mid + lo with hi = rn(x), mid = rn(x - hi),
 *     lo = rn(x - hi - mid); each subtraction is exact in float64.
 *
 *   MLP (3 hidden ReLU layers) forward, mean-squared-error loss, backward by
 *     the chain rule, and the Adam update with bias correction.
 *
 * Layouts:
 *   D     [F][N][N] row-major: D[(f*N + i)*N + j]
 *   u     element-major [E][N]: u[e*N + j];  node-major [N][E]: u[j*E + e]
 *   out   element-major [F][E][N]: out[(f*E + e)*N + i];
 *         node-major    [F][N][E]: out[(f*N + i)*E + e]
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The loop nest.  node_major selects the array layouts listed above.
 * nthreads <= 0 keeps the OpenMP default; 1 runs serially. */
void oracle_contract(const double *D, const double *u, double *out,
                     int64_t E, int32_t N, int32_t F, int32_t node_major,
                     int32_t nthreads)
{
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
    for (int64_t e = 0; e < E; ++e) {
        for (int32_t f = 0; f < F; ++f) {
            for (int32_t i = 0; i < N; ++i) {
                double acc = 0.0;
                for (int32_t j = 0; j < N; ++j) {
                    double d = D[((int64_t)f * N + i) * N + j];
                    double x = node_major ? u[(int64_t)j * E + e] : u[e * N + j];
                    acc += d * x;
                }
                if (node_major)
                    out[((int64_t)f * N + i) * E + e] = acc;
                else
                    out[((int64_t)f * E + e) * N + i] = acc;
            }
        }
    }
    (void)nthreads;
}

/* The volume derivative with per-element geometric factors (the dG FEM volume
 * workload of Table 1 with the chain rule applied inside the kernel):
 *
 *   out[d,e,i] = sum_f r[e,d,f] * ( sum_j D[f,i,j] * u[e,j] )
 *
 * over { [d,f,e,i,j] : 0<=d<Dd and 0<=f<F and 0<=e<E and 0<=i,j<N }: the inner sum
 * is the contraction above (the reference-coordinate derivative along f), the outer
 * one maps it to physical coordinate d with the element's factors r[e,d,:].
 * Layouts: element-major r [E][Dd][F], out [Dd][E][N];
 *          node-major    r [Dd][F][E], out [Dd][N][E]  (u as for the contraction). */
void oracle_contract_geo(const double *D, const double *u, const double *r, double *out,
                         int64_t E, int32_t N, int32_t F, int32_t Dd, int32_t node_major,
                         int32_t nthreads)
{
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
    for (int64_t e = 0; e < E; ++e) {
        for (int32_t d = 0; d < Dd; ++d) {
            for (int32_t i = 0; i < N; ++i) {
                double acc = 0.0;
                for (int32_t f = 0; f < F; ++f) {
                    double part = 0.0;
                    for (int32_t j = 0; j < N; ++j) {
                        double x = node_major ? u[(int64_t)j * E + e] : u[e * N + j];
                        part += D[((int64_t)f * N + i) * N + j] * x;
                    }
                    double g = node_major ? r[((int64_t)d * F + f) * E + e] : r[(e * Dd + d) * F + f];
                    acc += g * part;
                }
                if (node_major)
                    out[((int64_t)d * N + i) * E + e] = acc;
                else
                    out[((int64_t)d * E + e) * N + i] = acc;
            }
        }
    }
    (void)nthreads;
}

/* The surface part of the dG operator (the dG FEM surface workload of Table 1): at every
 * face node m of element e (face f = m / Nfp, node p = m % Nfp) the jump between the
 * interior trace u[e, fmask[f][p]] and the exterior trace, the value of u at global node
 * vmapP[e][m] (a neighbour's matching node; the element's own node on a boundary face),
 * scaled by the face's factor s[e][f]; the scaled jumps are lifted to the volume nodes:
 *
 *   out[e,i] (+)= sum_m L[i,m] * ( s[e, m / Nfp] * (u[e, fmask[m]] - u_flat[vmapP[e,m]]) )
 *
 * over { [e,i,m] : 0<=e<E and 0<=i<N and 0<=m<M }, M = Nf * Nfp.  Layouts: L [N][M],
 * fmask [M] (node of the element for face node m), vmapP [E][M] (index into u as a flat
 * array of E*N values), s [E][Nf], u and out element-major [E][N].  accumulate != 0 adds
 * to out, else overwrites it. */
void oracle_lift(const double *L, const int32_t *fmask, const int32_t *vmapP, const double *sc, const double *u,
                 double *out, int64_t E, int32_t N, int32_t Nf, int32_t Nfp, int32_t accumulate, int32_t nthreads)
{
    const int32_t M = Nf * Nfp;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
    for (int64_t e = 0; e < E; ++e) {
        for (int32_t i = 0; i < N; ++i) {
            double acc = 0.0;
            for (int32_t m = 0; m < M; ++m) {
                double jump = u[e * N + fmask[m]] - u[vmapP[e * M + m]];
                double flux = sc[e * Nf + m / Nfp] * jump;
                acc += L[(int64_t)i * M + m] * flux;
            }
            out[e * N + i] = accumulate ? out[e * N + i] + acc : acc;
        }
    }
    (void)nthreads;
}

/* Round one binary32 value to bfloat16, nearest-even, returned as a float.
 * The bfloat16 value is the upper half of a binary32 word; the lower 16 bits
 * decide the rounding: above half -> up, below -> down, exactly half -> to
 * the even upper half.  NaN stays NaN; a carry out of the mantissa moves into
 * the exponent, which is what rounding up to the next binade (or to infinity)
 * means. */
static float bf16_round_one(float x)
{
    uint32_t bits;
    memcpy(&bits, &x, 4);
    if ((bits & 0x7f800000u) == 0x7f800000u && (bits & 0x007fffffu) != 0) {
        bits |= 0x00400000u; /* quiet NaN */
        bits &= 0xffff0000u;
    } else {
        uint32_t upper = bits >> 16;
        uint32_t lower = bits & 0xffffu;
        if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u)))
            upper += 1u;
        bits = upper << 16;
    }
    float y;
    memcpy(&y, &bits, 4);
    return y;
}

void oracle_bf16_round(const float *x, float *y, int64_t n)
{
    for (int64_t k = 0; k < n; ++k)
        y[k] = bf16_round_one(x[k]);
}

/* Three-term bfloat16 split of each binary32 value. */
void oracle_bf16_split3(const float *x, float *hi, float *mid, float *lo, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) {
        double v = (double)x[k];
        float h = bf16_round_one(x[k]);
        double r1 = v - (double)h;           /* exact: fewer than 53 bits */
        float m = bf16_round_one((float)r1); /* r1 has <= 17 significant bits: exact in binary32 */
        double r2 = r1 - (double)m;
        float l = bf16_round_one((float)r2);
        hi[k] = h;
        mid[k] = m;
        lo[k] = l;
    }
}

/* ---------------------------------------------------------------------------
 * MLP cost model: y = w4 . h3 + b4, h_k = relu(W_k h_{k-1} + b_k), h_0 = x.
 * Parameter vector (float64), in this order:
 *   W1[H][din], b1[H], W2[H][H], b2[H], W3[H][H], b3[H], w4[H], b4[1]
 * ------------------------------------------------------------------------- */
int64_t oracle_mlp_param_count(int32_t din, int32_t H)
{
    return (int64_t)H * din + H + 2 * ((int64_t)H * H + H) + H + 1;
}

static void mlp_offsets(int32_t din, int32_t H, int64_t off[8])
{
    off[0] = 0;                          /* W1 */
    off[1] = off[0] + (int64_t)H * din;  /* b1 */
    off[2] = off[1] + H;                 /* W2 */
    off[3] = off[2] + (int64_t)H * H;    /* b2 */
    off[4] = off[3] + H;                 /* W3 */
    off[5] = off[4] + (int64_t)H * H;    /* b3 */
    off[6] = off[5] + H;                 /* w4 */
    off[7] = off[6] + H;                 /* b4 */
}

static void dense_relu(const double *W, const double *b, const double *in, double *pre,
                       double *out, int32_t nin, int32_t nout)
{
    for (int32_t o = 0; o < nout; ++o) {
        double s = b[o];
        for (int32_t k = 0; k < nin; ++k)
            s += W[(int64_t)o * nin + k] * in[k];
        pre[o] = s;
        out[o] = s > 0.0 ? s : 0.0;
    }
}

/* Forward pass for B samples x[B][din] -> y[B]. H <= 256. */
void oracle_mlp_forward(const double *p, const double *x, double *y, int64_t B, int32_t din,
                        int32_t H)
{
    int64_t off[8];
    double z1[256], a1[256], z2[256], a2[256], z3[256], a3[256];
    mlp_offsets(din, H, off);
    for (int64_t s = 0; s < B; ++s) {
        dense_relu(p + off[0], p + off[1], x + s * din, z1, a1, din, H);
        dense_relu(p + off[2], p + off[3], a1, z2, a2, H, H);
        dense_relu(p + off[4], p + off[5], a2, z3, a3, H, H);
        double out = p[off[7]];
        for (int32_t k = 0; k < H; ++k)
            out += p[off[6] + k] * a3[k];
        y[s] = out;
    }
}

/* Loss L = (1/B) sum_s (y_s - t_s)^2 and its gradient with respect to every
 * parameter, accumulated over the batch (chain rule, layer by layer).
 * Returns L; grad has oracle_mlp_param_count entries. */
double oracle_mlp_loss_grad(const double *p, const double *x, const double *t, int64_t B,
                            int32_t din, int32_t H, double *grad)
{
    int64_t off[8];
    double z1[256], a1[256], z2[256], a2[256], z3[256], a3[256];
    double g3[256], g2[256], g1[256];
    mlp_offsets(din, H, off);
    memset(grad, 0, sizeof(double) * (size_t)oracle_mlp_param_count(din, H));
    double loss = 0.0;
    for (int64_t s = 0; s < B; ++s) {
        const double *xs = x + s * din;
        dense_relu(p + off[0], p + off[1], xs, z1, a1, din, H);
        dense_relu(p + off[2], p + off[3], a1, z2, a2, H, H);
        dense_relu(p + off[4], p + off[5], a2, z3, a3, H, H);
        double y = p[off[7]];
        for (int32_t k = 0; k < H; ++k)
            y += p[off[6] + k] * a3[k];
        double r = y - t[s];
        loss += r * r;
        double dy = 2.0 * r / (double)B;     /* dL/dy_s */
        /* output layer */
        grad[off[7]] += dy;
        for (int32_t k = 0; k < H; ++k) {
            grad[off[6] + k] += dy * a3[k];
            g3[k] = dy * p[off[6] + k] * (z3[k] > 0.0 ? 1.0 : 0.0);  /* dL/dz3 */
        }
        /* layer 3: z3 = W3 a2 + b3 */
        for (int32_t o = 0; o < H; ++o) {
            grad[off[5] + o] += g3[o];
            for (int32_t k = 0; k < H; ++k)
                grad[off[4] + (int64_t)o * H + k] += g3[o] * a2[k];
        }
        for (int32_t k = 0; k < H; ++k) {
            double s2 = 0.0;
            for (int32_t o = 0; o < H; ++o)
                s2 += p[off[4] + (int64_t)o * H + k] * g3[o];
            g2[k] = s2 * (z2[k] > 0.0 ? 1.0 : 0.0);
        }
        /* layer 2: z2 = W2 a1 + b2 */
        for (int32_t o = 0; o < H; ++o) {
            grad[off[3] + o] += g2[o];
            for (int32_t k = 0; k < H; ++k)
                grad[off[2] + (int64_t)o * H + k] += g2[o] * a1[k];
        }
        for (int32_t k = 0; k < H; ++k) {
            double s1 = 0.0;
            for (int32_t o = 0; o < H; ++o)
                s1 += p[off[2] + (int64_t)o * H + k] * g2[o];
            g1[k] = s1 * (z1[k] > 0.0 ? 1.0 : 0.0);
        }
        /* layer 1: z1 = W1 x + b1 */
        for (int32_t o = 0; o < H; ++o) {
            grad[off[1] + o] += g1[o];
            for (int32_t k = 0; k < din; ++k)
                grad[off[0] + (int64_t)o * din + k] += g1[o] * xs[k];
        }
    }
    return loss / (double)B;
}

/* One Adam step (step counter t >= 1, bias-corrected moments). */
void oracle_adam_step(double *p, const double *g, double *m, double *v, int64_t n, int32_t t,
                      double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, (double)t);
    double c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        double mh = m[k] / c1;
        double vh = v[k] / c2;
        p[k] -= lr * mh / (sqrt(vh) + eps);
    }
}
