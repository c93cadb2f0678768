/*
 * tgp_oracle.c -- plain, slow CPU oracle for GP population evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path and includes nothing from it.
 *
 * What it computes (the plain definition the method must reach):
 *   for every tree t and every grid point (row, col), evaluate the expression
 *   tree recursively, then reduce each tree to its root-mean-squared error
 *   against the target:  RMSE_t = sqrt( (1/N) * sum_p (f_t(p) - P(p))^2 ).
 *
 * Passages followed (TensorGP, arXiv 2103.07512):
 *   - tensor phenotype over a fixed rank-2 grid of fitness cases: Sec. 3.1;
 *   - operator semantics and protections: Table 1 (add, sub, mult, div with
 *     0 on a zero denominator, sin, cos, neg, abs, min, max; and the rest of
 *     its mathematical and conditional operators: tan, exp, log with -1 for a
 *     negative argument, pow with 0 for 0^0, mdist, sqrt with 0 for a negative
 *     argument, sign, clip, mod, frac, if);
 *   - trigonometric operators take the argument multiplied by pi: Sec. 3.2
 *     (the default); the footnote of Table 1 states radians instead, which
 *     the `trig` argument selects (1: sin(a), cos(a), tan(a) of a itself);
 *   - Pagie polynomial target: Eq. 1;
 *   - RMSE fitness against the target: Sec. 4.1 and Table 2.
 *
 * Readings where the paper is silent or garbled:
 *   - Table 1 prints sin and cos swapped; the prose of Sec. 3.2 is followed:
 *     sin(a) := sin(pi*a), cos(a) := cos(pi*a).
 *   - The grid placement is not printed: inclusive linspace, x along columns,
 *     y along rows, flat index p = row*W + col, coordinates formed in IEEE
 *     binary32 as xlo + (float)col * ((xhi - xlo) / (float)(W - 1)) with no
 *     fused multiply-add; W == 1 gives x = xlo.  The oracle evaluates on these
 *     same float values widened to double.
 *   - Eq. 1 is undefined at 0 (x^-4); it is evaluated as x^4 / (1 + x^4), the
 *     continuous extension, which is 0 at x = 0.
 *   - RMSE divides by N.  A non-finite squared-error sum gives +inf.
 *   - Protected division returns 0 when the denominator equals 0 (either
 *     sign), otherwise the IEEE quotient.
 *   - min / max follow C fmin / fmax (a NaN operand yields the other one).
 *   - tan(a) := tan(pi*a) like sin and cos (Sec. 3.2 scales every
 *     trigonometric argument), computed as sin(pi*a) / cos(pi*a); +-inf where
 *     cos(pi*a) is exactly 0 (no protection is printed).
 *   - log(a) is -1 for a < 0 (printed) and the IEEE value otherwise, so
 *     log(0) = -inf; pow(a, b) is 0 for a = b = 0 (printed) and the IEEE
 *     pow otherwise (NaN for a negative base and a non-integer exponent);
 *     sqrt(a) is 0 for a < 0 (printed, arity 1: the printed 2 is a typo).
 *   - mdist(a, b) = (a + b) / 2; sign(a) in {-1, 0, 1} (NaN stays NaN);
 *     clip(x, y, z) = max(min(z, x), y) as printed; frac(a) = a - floor(a).
 *   - mod(a, b) is the floored remainder, a - b*floor(a/b), with the sign of
 *     b (no convention is printed; it is Python's and the one that keeps
 *     frac(a) = mod(a, 1)); NaN for b = 0 (no protection is printed).
 *   - if(c, a, b) is a where c != 0 (NaN counts as true), b where c == 0.
 *
 * Two evaluation modes run side by side on every node:
 *   - FP64: every node in binary64;
 *   - FP32-faithful: every node computed in binary64 from binary32 operands and
 *     rounded to binary32 before its parent uses it.  For + - * / this is the
 *     correctly rounded binary32 result; for sin/cos it is the (almost always)
 *     correctly rounded value of sin(pi*a).
 * Per element the oracle flags near-singular division: some div node of the
 * tree saw a denominator with |b| < 1e-6 in either mode.
 *
 * Per element it also bounds how far ANY binary32 evaluation of the tree can
 * land from the exact value, given operators that are correctly rounded for
 * + - * / (error <= u|r|, u = 2^-24, plus 2^-149 in the subnormal range) and
 * sin/cos(pi*a) within 2 ulp of the exact value of the binary32 argument.
 * It is a forward running-error bound, propagated node by node with the
 * binary64 values standing in for the exact ones:
 *   x, y, const: 0 (binary32 values, exact)
 *   a +- b:  P = Ea + Eb
 *   a * b:   P = |b|Ea + |a|Eb + EaEb
 *   a / b:   P = (Ea + |a/b| Eb) / (|b| - Eb), unbounded if |b| <= Eb (the
 *            sign or zero test of the denominator is then undecided); 0 for
 *            an exact zero denominator (the protected result is exactly 0)
 *   sin(pi a): P = min(pi Ea |cos(pi a)| + (pi Ea)^2 / 2, 2) (Taylor's
 *            theorem: the first derivative at a, and |second| <= pi^2 on the
 *            interval); cos(pi a) likewise with |sin(pi a)|; plus 2 ulp of
 *            the result (radians: pi replaced by 1; tan likewise)
 *   -a, |a|: Ea;  min/max: the error of the operand taken when the two are
 *            further apart than Ea + Eb (the comparison is then decided),
 *            else max(Ea, Eb)
 *   tan(pi a): P = pi Ea / (|c| - pi Ea)^2 with c = cos(pi a), unbounded if
 *            |c| <= pi Ea; plus 4 ulp (a quotient of two trig values)
 *   exp(a): P = |v| (e^Ea - 1), plus 2 ulp
 *   log(a): a > 0: P = log(a / (a - Ea)), unbounded if a <= Ea; a < 0: 0,
 *            unbounded if a + Ea >= 0; plus 2 ulp
 *   pow(a, b): exact operands: 8 ulp; otherwise a > Ea: with L = log(a/(a-Ea))
 *            and M = max|log(a +- Ea)|, P = |v| (e^(|b| L + Eb M + Eb L) - 1)
 *            plus 8 ulp; unbounded for a <= Ea
 *   mdist(a, b): P = (Ea + Eb) / 2 plus one rounding; unbounded if the sum
 *            may overflow
 *   sqrt(a): a - Ea >= 0: P = sqrt(a) - sqrt(a - Ea); else P = sqrt(max(a,0)
 *            + Ea); plus one rounding
 *   sign(a): 0, unbounded when the interval a +- Ea holds 0 and Ea > 0
 *   clip: max(Ex, Ey, Ez) (min and max)
 *   mod(a, b): exact operands: one rounding; otherwise unbounded unless b is
 *            away from 0 and floor(a/b) is the same over the operand box, then
 *            P = Ea + |floor(a/b)| Eb plus one rounding
 *   frac(a): P = Ea plus one rounding, unbounded if a +- Ea holds an integer
 *            other than at a exact a
 *   if(c, a, b): the chosen operand's bound; unbounded if c +- Ec holds 0 and
 *            Ec > 0
 * and E = P + u(|v| + P) (+ 2^-150 for a possibly subnormal product or
 * quotient); unbounded once |v| + E reaches the binary32 range.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -o liboracle.so tgp_oracle.c -lm
 * (-ffp-contract=off keeps a*b+c from being fused, which some targets do by
 * default and which would change the binary32 grid coordinates.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* pi to binary64 precision */
#define ORACLE_PI 3.14159265358979323846

/* Opcodes of the token stream: the three terminals x, y and an ephemeral
 * constant, the 10 functions of the configured set, then the rest of the
 * mathematical and conditional operators of Table 1. */
enum {
    O_X = 0, O_Y = 1, O_CONST = 2,
    O_ADD = 3, O_SUB = 4, O_MUL = 5, O_DIV = 6,
    O_SIN = 7, O_COS = 8, O_NEG = 9, O_ABS = 10, O_MIN = 11, O_MAX = 12,
    O_TAN = 13, O_EXP = 14, O_LOG = 15, O_POW = 16, O_MDIST = 17, O_SQRT = 18,
    O_SIGN = 19, O_CLIP = 20, O_MOD = 21, O_FRAC = 22, O_IF = 23,
    O_COUNT = 24
};

enum { ORD_PREFIX = 0, ORD_POSTFIX = 1 };

/* error codes returned by the oracle */
enum { OR_OK = 0, OR_BAD_OPCODE = -1, OR_MALFORMED = -2, OR_IMM = -3, OR_ARG = -4, OR_NOMEM = -5 };

static int arity_of(int op)
{
    switch (op) {
    case O_X: case O_Y: case O_CONST: return 0;
    case O_SIN: case O_COS: case O_NEG: case O_ABS:
    case O_TAN: case O_EXP: case O_LOG: case O_SQRT: case O_SIGN: case O_FRAC: return 1;
    case O_ADD: case O_SUB: case O_MUL: case O_DIV: case O_MIN: case O_MAX:
    case O_POW: case O_MDIST: case O_MOD: return 2;
    case O_CLIP: case O_IF: return 3;
    default: return -1;
    }
}

/* one parsed tree node */
typedef struct {
    int op;
    int kid[3];     /* indices into the same node array, -1 if absent */
    double imm;     /* the constant, as the binary32 value widened */
} onode;

/* ---------------------------------------------------------------- parsing */

/* Prefix: the operator precedes its operands (recursive descent). */
static int parse_prefix(const int32_t* ops, int64_t n_tok, const float* imm, int64_t n_imm,
                        int64_t* tok_pos, int64_t* imm_pos, onode* nodes, int* n_nodes, int* out)
{
    if (*tok_pos >= n_tok) return OR_MALFORMED;
    int op = ops[(*tok_pos)++];
    int ar = arity_of(op);
    if (ar < 0) return OR_BAD_OPCODE;
    int me = (*n_nodes)++;
    nodes[me].op = op;
    nodes[me].kid[0] = nodes[me].kid[1] = nodes[me].kid[2] = -1;
    nodes[me].imm = 0.0;
    if (op == O_CONST) {
        if (*imm_pos >= n_imm) return OR_IMM;
        nodes[me].imm = (double)imm[(*imm_pos)++];
    }
    for (int c = 0; c < ar; c++) {
        int k;
        int rc = parse_prefix(ops, n_tok, imm, n_imm, tok_pos, imm_pos, nodes, n_nodes, &k);
        if (rc) return rc;
        nodes[me].kid[c] = k;
    }
    *out = me;
    return OR_OK;
}

/* Postfix: operands precede their operator (explicit stack). */
static int parse_postfix(const int32_t* ops, int64_t n_tok, const float* imm, int64_t n_imm,
                         int64_t* imm_pos, onode* nodes, int* out)
{
    int* stack = (int*)malloc(sizeof(int) * (size_t)(n_tok + 1));
    if (!stack) return OR_NOMEM;
    int sp = 0, n = 0, rc = OR_OK;
    for (int64_t i = 0; i < n_tok; i++) {
        int op = ops[i];
        int ar = arity_of(op);
        if (ar < 0) { rc = OR_BAD_OPCODE; break; }
        if (sp < ar) { rc = OR_MALFORMED; break; }
        int me = n++;
        nodes[me].op = op;
        nodes[me].kid[0] = nodes[me].kid[1] = nodes[me].kid[2] = -1;
        nodes[me].imm = 0.0;
        if (op == O_CONST) {
            if (*imm_pos >= n_imm) { rc = OR_IMM; break; }
            nodes[me].imm = (double)imm[(*imm_pos)++];
        }
        for (int c = ar - 1; c >= 0; c--) nodes[me].kid[c] = stack[--sp];
        stack[sp++] = me;
    }
    if (rc == OR_OK && sp != 1) rc = OR_MALFORMED;
    if (rc == OR_OK) *out = stack[0];
    free(stack);
    return rc;
}

typedef struct {
    onode* nodes;
    int root;
} otree;

/* Parses every tree of a population.  imm is consumed in stream order across
 * all trees.  On success trees[t] holds malloc'ed node arrays. */
static int parse_population(const int32_t* ops, const float* imm, int64_t n_imm,
                            const int64_t* tree_off, int32_t n_trees, int32_t order, otree* trees)
{
    int64_t imm_pos = 0;
    for (int32_t t = 0; t < n_trees; t++) trees[t].nodes = NULL;
    for (int32_t t = 0; t < n_trees; t++) {
        int64_t n_tok = tree_off[t + 1] - tree_off[t];
        if (n_tok <= 0) return OR_MALFORMED;
        trees[t].nodes = (onode*)malloc(sizeof(onode) * (size_t)n_tok);
        if (!trees[t].nodes) return OR_NOMEM;
        const int32_t* tk = ops + tree_off[t];
        int rc;
        if (order == ORD_PREFIX) {
            int64_t pos = 0;
            int n = 0;
            rc = parse_prefix(tk, n_tok, imm, n_imm, &pos, &imm_pos, trees[t].nodes, &n, &trees[t].root);
            if (rc == OR_OK && pos != n_tok) rc = OR_MALFORMED;
        } else if (order == ORD_POSTFIX) {
            rc = parse_postfix(tk, n_tok, imm, n_imm, &imm_pos, trees[t].nodes, &trees[t].root);
        } else {
            rc = OR_ARG;
        }
        if (rc) return rc;
    }
    if (imm_pos != n_imm) return OR_IMM;
    return OR_OK;
}

static void free_population(otree* trees, int32_t n_trees)
{
    for (int32_t t = 0; t < n_trees; t++) free(trees[t].nodes);
}

/* ------------------------------------------------------------ arithmetic */

/* sin(pi*a) for a binary64 a.  The argument is reduced exactly: r = a mod 2,
 * n = nearest integer to 2r, f = r - n/2 in [-1/4, 1/4] (both steps are exact
 * in binary64), then the quadrant identity picks sin or cos of pi*f.  This
 * gives exact zeros at integers and exact +-1 at half-integers. */
double oracle_sinpi(double a)
{
    if (!isfinite(a)) return NAN;
    double r = fmod(a, 2.0);
    double n = nearbyint(2.0 * r);
    double f = r - 0.5 * n;
    int q = (int)fmod(n, 4.0);
    if (q < 0) q += 4;
    double pf = ORACLE_PI * f, v;
    switch (q) {
    case 0: v = sin(pf); break;
    case 1: v = cos(pf); break;
    case 2: v = -sin(pf); break;
    default: v = -cos(pf); break;
    }
    return v == 0.0 ? 0.0 : v;   /* zeros are returned as +0 */
}

/* cos(pi*a), same reduction. */
double oracle_cospi(double a)
{
    if (!isfinite(a)) return NAN;
    double r = fmod(a, 2.0);
    double n = nearbyint(2.0 * r);
    double f = r - 0.5 * n;
    int q = (int)fmod(n, 4.0);
    if (q < 0) q += 4;
    double pf = ORACLE_PI * f, v;
    switch (q) {
    case 0: v = cos(pf); break;
    case 1: v = -sin(pf); break;
    case 2: v = -cos(pf); break;
    default: v = sin(pf); break;
    }
    return v == 0.0 ? 0.0 : v;   /* zeros are returned as +0 */
}

/* Table 1, div: x/y, and 0 when the denominator is 0. */
static double pdiv(double a, double b)
{
    if (b == 0.0) return 0.0;
    return a / b;
}

/* Table 1, log: -1 for a negative argument. */
static double plog(double a)
{
    if (a < 0.0) return -1.0;
    return log(a);
}

/* Table 1, pow: 0 when both operands are 0. */
static double ppow(double a, double b)
{
    if (a == 0.0 && b == 0.0) return 0.0;
    return pow(a, b);
}

/* Table 1, sqrt: 0 for a negative argument. */
static double psqrt(double a)
{
    if (a < 0.0) return 0.0;
    return sqrt(a);
}

static double sign_of(double a)
{
    if (a > 0.0) return 1.0;
    if (a < 0.0) return -1.0;
    if (a == 0.0) return 0.0;
    return a;   /* NaN */
}

/* floored remainder a - b*floor(a/b), with the sign of b */
static double floor_mod(double a, double b)
{
    double r = fmod(a, b);
    if (r != 0.0 && ((r < 0.0) != (b < 0.0))) r += b;
    return r;
}

/* One operator of Table 1 applied in binary64 (c: third operand; rad:
 * trigonometric arguments in radians instead of multiplied by pi). */
static double apply64(int op, double a, double b, double c, int rad)
{
    switch (op) {
    case O_TAN: return rad ? tan(a) : oracle_sinpi(a) / oracle_cospi(a);
    case O_EXP: return exp(a);
    case O_LOG: return plog(a);
    case O_POW: return ppow(a, b);
    case O_MDIST: return (a + b) / 2.0;
    case O_SQRT: return psqrt(a);
    case O_SIGN: return sign_of(a);
    case O_CLIP: return fmax(fmin(c, a), b);
    case O_MOD: return floor_mod(a, b);
    case O_FRAC: return a - floor(a);
    case O_IF: return a != 0.0 ? b : c;   /* NaN != 0 is true */
    case O_ADD: return a + b;
    case O_SUB: return a - b;
    case O_MUL: return a * b;
    case O_DIV: return pdiv(a, b);
    case O_SIN: return rad ? sin(a) : oracle_sinpi(a);
    case O_COS: return rad ? cos(a) : oracle_cospi(a);
    case O_NEG: return -a;
    case O_ABS: return fabs(a);
    case O_MIN: return fmin(a, b);
    case O_MAX: return fmax(a, b);
    default: return NAN;
    }
}

#define NEAR_SINGULAR 1e-6

#define U32 5.9604644775390625e-08          /* 2^-24, unit roundoff of binary32 */
#define TINY32 1.4012984643248171e-45       /* 2^-149, smallest binary32 subnormal */
#define MAX32 3.4028234663852886e+38        /* largest finite binary32 */
#define TRIG_ULPS 2.0

#define MIN_NORMAL32 1.1754943508222875e-38   /* 2^-126 */

/* Rounding error of one binary32 operation whose computed result lies within
 * `prop` of v: at most u * |computed| <= u * (|v| + prop), plus half the
 * subnormal spacing when the result may be subnormal.  A sum or difference is
 * exact in the subnormal range, so `exact_sub` drops that term; a result that
 * is exactly zero from exact operands is exact. */
static double rnd32(double v, double prop, int exact_sub)
{
    double m = fabs(v) + prop;
    if (m == 0.0) return 0.0;
    double e = U32 * m;
    if (!exact_sub && m < MIN_NORMAL32) e += 0.5 * TINY32;
    return e;
}

#define TAN_ULPS 4.0
#define EXP_ULPS 2.0
#define LOG_ULPS 2.0
#define POW_ULPS 8.0

/* k ulps of a binary32 result of magnitude up to m (ulp <= 2u|r|, and the
 * subnormal spacing). */
static double ulps32(double k, double m)
{
    return k * (2.0 * U32 * m + TINY32);
}

/* Error bound of one node from its operands' bounds (see the header). */
static double err_bound(int op, double a, double b, double c, double ea, double eb, double ec, double v, int rad)
{
    const double k = rad ? 1.0 : ORACLE_PI;   /* d(argument)/da of the trigonometric operators */
    double e, prop;
    if (op == O_IF) {   /* only the chosen operand matters, once the zero test is decided */
        if (!isfinite(v) || !isfinite(ea)) return INFINITY;
        if (ea > 0.0 && fabs(a) <= ea) return INFINITY;
        e = a != 0.0 ? eb : ec;
        if (!isfinite(e) || fabs(v) + e >= MAX32) return INFINITY;
        return e;
    }
    if (!isfinite(v) || !isfinite(ea) || !isfinite(eb) || !isfinite(ec)) return INFINITY;
    switch (op) {
    case O_TAN: {
        double cs = fabs(rad ? cos(a) : oracle_cospi(a));
        if (cs <= k * ea) return INFINITY;
        double d = cs - k * ea;
        prop = k * ea / (d * d);
        e = prop + ulps32(TAN_ULPS, fabs(v) + prop);
        break;
    }
    case O_EXP:
        prop = fabs(v) * expm1(ea);
        e = prop + ulps32(EXP_ULPS, fabs(v) + prop);
        break;
    case O_LOG:
        if (a > 0.0) {
            if (a <= ea) return INFINITY;
            prop = log(a / (a - ea));
        } else if (a < 0.0) {
            if (a + ea >= 0.0) return INFINITY;
            prop = 0.0;
        } else {
            return INFINITY;   /* log(0) = -inf */
        }
        e = prop + (a < 0.0 ? 0.0 : ulps32(LOG_ULPS, fabs(v) + prop));
        break;
    case O_POW:
        if (ea == 0.0 && eb == 0.0) {
            e = (a == 0.0 && b == 0.0) ? 0.0 : ulps32(POW_ULPS, fabs(v));
            break;
        }
        if (a <= ea) return INFINITY;
        {
            double L = log(a / (a - ea));
            double M = fmax(fabs(log(a - ea)), fabs(log(a + ea)));
            prop = fabs(v) * expm1(fabs(b) * L + eb * M + eb * L);
        }
        e = prop + ulps32(POW_ULPS, fabs(v) + prop);
        break;
    case O_MDIST:
        if (fabs(a) + fabs(b) + ea + eb >= MAX32) return INFINITY;   /* the binary32 sum may overflow */
        prop = 0.5 * (ea + eb);
        e = prop + rnd32(v, prop, 0);
        break;
    case O_SQRT:
        if (a - ea >= 0.0) prop = sqrt(a) - sqrt(a - ea);
        else prop = sqrt(fmax(a, 0.0) + ea);
        e = prop + rnd32(v, prop, 0);
        break;
    case O_SIGN:
        if (ea > 0.0 && fabs(a) <= ea) return INFINITY;
        e = 0.0;
        break;
    case O_CLIP:
        e = fmax(ea, fmax(eb, ec));
        break;
    case O_MOD: {
        if (ea == 0.0 && eb == 0.0) {
            e = rnd32(v, 0.0, 1);
            break;
        }
        if (fabs(b) <= eb) return INFINITY;
        double q1 = (a - ea) / (b - eb), q2 = (a - ea) / (b + eb);
        double q3 = (a + ea) / (b - eb), q4 = (a + ea) / (b + eb);
        double k = floor(a / b);
        if (floor(q1) != k || floor(q2) != k || floor(q3) != k || floor(q4) != k) return INFINITY;
        prop = ea + fabs(k) * eb;
        e = prop + rnd32(v, prop, 1);
        break;
    }
    case O_FRAC:
        if (ea > 0.0 && floor(a - ea) != floor(a + ea)) return INFINITY;
        prop = ea;
        e = prop + rnd32(v, prop, 1);
        break;

    case O_ADD: case O_SUB:
        prop = ea + eb;
        e = prop + rnd32(v, prop, 1);
        break;
    case O_MUL:
        prop = fabs(b) * ea + fabs(a) * eb + ea * eb;
        e = prop + rnd32(v, prop, 0);
        break;
    case O_DIV:
        if (b == 0.0 && eb == 0.0) { e = 0.0; break; }   /* exact zero denominator: result 0 */
        if (fabs(b) <= eb) return INFINITY;
        prop = (ea + fabs(a / b) * eb) / (fabs(b) - eb);
        e = prop + rnd32(v, prop, 0);
        break;
    case O_SIN: case O_COS: {
        /* |derivative| at a, over k: |cos| for sin, |sin| for cos */
        double slope = op == O_SIN ? fabs(rad ? cos(a) : oracle_cospi(a)) : fabs(rad ? sin(a) : oracle_sinpi(a));
        prop = fmin(k * ea * slope + 0.5 * (k * ea) * (k * ea), 2.0);
        e = prop + TRIG_ULPS * (2.0 * U32 * (fabs(v) + prop) + TINY32);
        break;
    }
    case O_NEG: case O_ABS:
        e = ea;
        break;
    case O_MIN: case O_MAX:
        if (fabs(a - b) > ea + eb) e = (v == a) ? ea : eb;   /* decided comparison: the taken operand */
        else e = fmax(ea, eb);
        break;
    default:
        return INFINITY;
    }
    if (fabs(v) + e >= MAX32) return INFINITY;
    return e;
}

typedef struct {
    double x64, y64;   /* coordinates (binary32 values widened) */
    int flag;          /* near-singular division seen */
    int rad;           /* trigonometric arguments in radians */
} opoint;

/* Recursive tree walk in both modes at once, with the error bound. */
static void eval_node(const onode* nodes, int i, opoint* pt, double* v64, float* v32, double* eb)
{
    const onode* n = &nodes[i];
    switch (n->op) {
    case O_X: *v64 = pt->x64; *v32 = (float)pt->x64; *eb = 0.0; return;
    case O_Y: *v64 = pt->y64; *v32 = (float)pt->y64; *eb = 0.0; return;
    case O_CONST: *v64 = n->imm; *v32 = (float)n->imm; *eb = 0.0; return;
    default: break;
    }
    double a64 = 0.0, b64 = 0.0, c64 = 0.0, ea = 0.0, eb_ = 0.0, ec = 0.0;
    float a32 = 0.0f, b32 = 0.0f, c32 = 0.0f;
    eval_node(nodes, n->kid[0], pt, &a64, &a32, &ea);
    if (n->kid[1] >= 0) eval_node(nodes, n->kid[1], pt, &b64, &b32, &eb_);
    if (n->kid[2] >= 0) eval_node(nodes, n->kid[2], pt, &c64, &c32, &ec);
    if (n->op == O_DIV) {
        if (fabs(b64) < NEAR_SINGULAR || fabs((double)b32) < NEAR_SINGULAR) pt->flag = 1;
    }
    *v64 = apply64(n->op, a64, b64, c64, pt->rad);
    *v32 = (float)apply64(n->op, (double)a32, (double)b32, (double)c32, pt->rad);
    *eb = err_bound(n->op, a64, b64, c64, ea, eb_, ec, *v64, pt->rad);
}

/* ------------------------------------------------------------------ grid */

/* Coordinate of column col (or row) on an inclusive linspace of n points,
 * formed in binary32 exactly as the grid reading states. */
static float grid_coord(float lo, float hi, int32_t n, int64_t i)
{
    if (n <= 1) return lo;
    float step = (hi - lo) / (float)(n - 1);
    float prod = (float)i * step;
    return lo + prod;
}

void oracle_grid_point(int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi,
                       int64_t p, float* x, float* y)
{
    int64_t row = p / W, col = p % W;
    *x = grid_coord(xlo, xhi, W, col);
    *y = grid_coord(ylo, yhi, H, row);
}

/* Eq. 1, Pagie polynomial, written as x^4/(1+x^4) + y^4/(1+y^4) (continuous
 * extension at 0). */
double oracle_pagie(double x, double y)
{
    double x4 = x * x * x * x;
    double y4 = y * y * y * y;
    return x4 / (1.0 + x4) + y4 / (1.0 + y4);
}

/* ------------------------------------------------------------ public API */

/*
 * Evaluates every tree of a population at n_pts grid points (flat indices in
 * pts, or all H*W points in order when pts == NULL).
 *   out64 [n_trees][n_pts]  binary64 values (required)
 *   out32 [n_trees][n_pts]  FP32-faithful values (may be NULL)
 *   flags [n_trees][n_pts]  1 where a division saw |denominator| < 1e-6 (may be NULL)
 *   errb  [n_trees][n_pts]  bound on |any binary32 evaluation - exact| (may be NULL)
 * trig: 0 = trigonometric arguments multiplied by pi (Sec. 3.2), 1 = radians.
 * Returns 0 or a negative error code (malformed tokens, bad opcode, imm count).
 */
int oracle_eval(const int32_t* ops, const float* imm, int64_t n_imm, const int64_t* tree_off,
                int32_t n_trees, int32_t order,
                int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi,
                int64_t n_pts, const int64_t* pts,
                double* out64, float* out32, uint8_t* flags, double* errb, int32_t trig)
{
    if (n_trees < 0 || W <= 0 || H <= 0 || n_pts < 0 || (trig != 0 && trig != 1)) return OR_ARG;
    otree* trees = (otree*)calloc((size_t)(n_trees > 0 ? n_trees : 1), sizeof(otree));
    if (!trees) return OR_NOMEM;
    int rc = parse_population(ops, imm, n_imm, tree_off, n_trees, order, trees);
    if (rc) { free_population(trees, n_trees); free(trees); return rc; }
    for (int32_t t = 0; t < n_trees; t++) {
        for (int64_t i = 0; i < n_pts; i++) {
            int64_t p = pts ? pts[i] : i;
            float xf, yf;
            oracle_grid_point(W, H, xlo, xhi, ylo, yhi, p, &xf, &yf);
            opoint pt = { (double)xf, (double)yf, 0, trig };
            double v64, e;
            float v32;
            eval_node(trees[t].nodes, trees[t].root, &pt, &v64, &v32, &e);
            out64[(size_t)t * n_pts + i] = v64;
            if (out32) out32[(size_t)t * n_pts + i] = v32;
            if (flags) flags[(size_t)t * n_pts + i] = (uint8_t)pt.flag;
            if (errb) errb[(size_t)t * n_pts + i] = e;
        }
    }
    free_population(trees, n_trees);
    free(trees);
    return OR_OK;
}

/* target kinds */
enum { TG_PAGIE = 0, TG_VALUES = 1 };

/*
 * RMSE of every tree against the target over all H*W points (or over the
 * n_pts points listed in pts, dividing by n_pts).
 *   target_kind 0: Pagie polynomial (Eq. 1) at the grid's coordinates;
 *   target_kind 1: target_vals[p] (binary64, indexed by flat point index).
 *   rmse64 [n_trees]: RMSE of the binary64 phenotype;
 *   rmse32 [n_trees]: RMSE of the FP32-faithful phenotype (may be NULL);
 *   n_flagged [n_trees]: points with a near-singular division (may be NULL);
 *   rmse_err [n_trees]: sqrt(mean(E^2)) of the per-element error bounds, a
 *     bound on how far the RMSE of any binary32 evaluation of the phenotype
 *     can be from rmse64 (triangle inequality in the L2 norm); +inf when
 *     some element is unbounded (may be NULL).
 * trig as for oracle_eval.  A non-finite sum gives +inf.
 */
int oracle_fitness(const int32_t* ops, const float* imm, int64_t n_imm, const int64_t* tree_off,
                   int32_t n_trees, int32_t order,
                   int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi,
                   int32_t target_kind, const double* target_vals,
                   int64_t n_pts, const int64_t* pts,
                   double* rmse64, double* rmse32, int64_t* n_flagged, double* rmse_err, int32_t trig)
{
    if (n_trees < 0 || W <= 0 || H <= 0 || (trig != 0 && trig != 1)) return OR_ARG;
    if (target_kind == TG_VALUES && !target_vals) return OR_ARG;
    if (target_kind != TG_PAGIE && target_kind != TG_VALUES) return OR_ARG;
    int64_t N = pts ? n_pts : (int64_t)W * (int64_t)H;
    otree* trees = (otree*)calloc((size_t)(n_trees > 0 ? n_trees : 1), sizeof(otree));
    if (!trees) return OR_NOMEM;
    int rc = parse_population(ops, imm, n_imm, tree_off, n_trees, order, trees);
    if (rc) { free_population(trees, n_trees); free(trees); return rc; }
    for (int32_t t = 0; t < n_trees; t++) {
        double s64 = 0.0, s32 = 0.0, se = 0.0;
        int64_t nf = 0;
        for (int64_t i = 0; i < N; i++) {
            int64_t p = pts ? pts[i] : i;
            float xf, yf;
            oracle_grid_point(W, H, xlo, xhi, ylo, yhi, p, &xf, &yf);
            double tv = target_kind == TG_PAGIE ? oracle_pagie((double)xf, (double)yf) : target_vals[p];
            opoint pt = { (double)xf, (double)yf, 0, trig };
            double v64, e;
            float v32;
            eval_node(trees[t].nodes, trees[t].root, &pt, &v64, &v32, &e);
            double d64 = v64 - tv;
            double d32 = (double)v32 - tv;
            s64 += d64 * d64;
            s32 += d32 * d32;
            se += e * e;
            nf += pt.flag;
        }
        double r64 = sqrt(s64 / (double)N);
        double r32 = sqrt(s32 / (double)N);
        rmse64[t] = isfinite(r64) ? r64 : INFINITY;
        if (rmse32) rmse32[t] = isfinite(r32) ? r32 : INFINITY;
        if (n_flagged) n_flagged[t] = nf;
        if (rmse_err) {
            double re = sqrt(se / (double)N);
            rmse_err[t] = isfinite(re) ? re : INFINITY;
        }
    }
    free_population(trees, n_trees);
    free(trees);
    return OR_OK;
}

/*
 * Sums behind the fitness comparison, split by how each element can be
 * compared with a binary32 evaluation.  An element is "comparable" when its
 * error bound is finite (every zero or sign test on its path is decided; a
 * near-singular denominator is then harmless) and the FP32-faithful value
 * lies within tol * (1 + |v64|) of the binary64 one (else binary32
 * evaluation is ill-conditioned there); the others are listed.  Sums rather than RMSE
 * values are returned so that the caller may split the points into chunks
 * and add.
 *   sums [n_trees][8]:
 *     0  sum over all points of (v64 - target)^2
 *     1  sum over all points of (v32 - target)^2
 *     2  sum over comparable points of (v64 - target)^2
 *     3  sum over comparable points of (v32 - target)^2
 *     4  sum over comparable points of E^2 (E the element's error bound)
 *     5  number of comparable points
 *     6  number of points with a near-singular division (comparable or not)
 *     7  number of points that are not comparable
 *   ex_tree, ex_pt [ex_cap]: (tree, flat point index) of every element that is
 *     not comparable, in tree-then-point order; ex_n receives their count
 *     (the lists hold the first ex_cap of them; NULL with ex_cap 0 to count).
 * Targets and trig as for oracle_fitness.
 */
int oracle_fitness_parts(const int32_t* ops, const float* imm, int64_t n_imm, const int64_t* tree_off,
                         int32_t n_trees, int32_t order,
                         int32_t W, int32_t H, float xlo, float xhi, float ylo, float yhi,
                         int32_t target_kind, const double* target_vals,
                         int64_t n_pts, const int64_t* pts, int32_t trig, double tol,
                         double* sums, int32_t* ex_tree, int64_t* ex_pt, int64_t ex_cap, int64_t* ex_n)
{
    if (n_trees < 0 || W <= 0 || H <= 0 || (trig != 0 && trig != 1) || !sums || !ex_n) return OR_ARG;
    if (target_kind == TG_VALUES && !target_vals) return OR_ARG;
    if (target_kind != TG_PAGIE && target_kind != TG_VALUES) return OR_ARG;
    int64_t N = pts ? n_pts : (int64_t)W * (int64_t)H;
    otree* trees = (otree*)calloc((size_t)(n_trees > 0 ? n_trees : 1), sizeof(otree));
    if (!trees) return OR_NOMEM;
    int rc = parse_population(ops, imm, n_imm, tree_off, n_trees, order, trees);
    if (rc) { free_population(trees, n_trees); free(trees); return rc; }
    int64_t nx = 0;
    for (int32_t t = 0; t < n_trees; t++) {
        double* s = sums + (size_t)t * 8;
        for (int k = 0; k < 8; k++) s[k] = 0.0;
        for (int64_t i = 0; i < N; i++) {
            int64_t p = pts ? pts[i] : i;
            float xf, yf;
            oracle_grid_point(W, H, xlo, xhi, ylo, yhi, p, &xf, &yf);
            double tv = target_kind == TG_PAGIE ? oracle_pagie((double)xf, (double)yf) : target_vals[p];
            opoint pt = { (double)xf, (double)yf, 0, trig };
            double v64, e;
            float v32;
            eval_node(trees[t].nodes, trees[t].root, &pt, &v64, &v32, &e);
            double d64 = v64 - tv, d32 = (double)v32 - tv;
            s[0] += d64 * d64;
            s[1] += d32 * d32;
            int ok32 = (double)v32 == v64 || fabs((double)v32 - v64) <= tol * (1.0 + fabs(v64));
            s[6] += pt.flag;
            if (isfinite(e) && ok32) {
                s[2] += d64 * d64;
                s[3] += d32 * d32;
                s[4] += e * e;
                s[5] += 1.0;
            } else {
                s[7] += 1.0;
                if (nx < ex_cap) { ex_tree[nx] = t; ex_pt[nx] = p; }
                nx++;
            }
        }
    }
    *ex_n = nx;
    free_population(trees, n_trees);
    free(trees);
    return OR_OK;
}

/* Arity of an opcode (-1 if unknown); exported for the tests' brute force. */
int oracle_arity(int32_t op) { return arity_of(op); }
