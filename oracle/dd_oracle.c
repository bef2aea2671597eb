/*
 * Plain CPU oracle for incoherent dedispersion (Barsdell, Bailes, Barnes &
 * Fluke, "Accelerating incoherent dedispersion", arXiv:1201.5380).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference legs use it.  It shares no code, header, table or
 * constant with the CUDA library; both sides are written from the paper.
 *
 * Every routine is the slow, literal form of the definition it cites:
 *   - partial delay, Eq. 3 (eq:partial_delay), and integer delay, Eq. 4
 *     (eq:delay), in IEEE double, with round() read as round-half-up;
 *   - the direct transform, Eq. 2 (eq:direct), summed per (d, t) over
 *     channels in channel order, exact in 64-bit integers for integer input
 *     and in double for 32-bit float input;
 *   - sub-band dedispersion, Sec. 4.1 (two direct passes: sub-bands at
 *     nominal DMs, then a direct pass over sub-bands, the stage-2 shift being
 *     the sum of Eq. (eq:combining_subbands), which telescopes to the delay of
 *     the sub-band's first channel);
 *   - the sub-band smearing bound of Appendix B (eq:subband_smear_approx,
 *     eq:RelativeSmearingSubband);
 *   - tree dedispersion, Sec. 3.1 (Eq. tree_algorithm_first .. last with the
 *     delay Theta of Eq. tree_integer_delay and the shuffle Phi of Eq.
 *     shuffle, step by step), and the piecewise linear tree method of Sec.
 *     3.1.1 (the tree per sub-band, Eq. subband_result, then Eq.
 *     combining_subbands), with its DM limit (Eq. tree_dm_limit) and the
 *     smear bound of Appendix A (Eq. subband_error);
 *   - the trial-DM list: the paper only says it bounds the smearing due to
 *     a wrong trial DM (Sec. 5.2, after Cordes & McLaughlin 2003); the
 *     recurrence below is this project's reading of that rule (see
 *     orc_dm_list).
 *
 * Input layout (the paper does not fix an external format; Sec. 2.3 only
 * says samples narrower than a word are packed and unpacked by shift and
 * mask): a time-major filterbank, row t holding channels 0..nchans-1; with
 * nbits < 8 channel c occupies bits [(c*nbits) mod 8, +nbits) of byte
 * (c*nbits)/8 of the row, least significant bits first; samples unsigned.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -ffp-contract=off (no FMA
 * contraction, so that the double-precision delay evaluation rounds the same
 * way on every host).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Dispersion constant of Eq. 1, MHz^2 pc^-1 cm^3 s (Sec. 1). */
static const double ORC_K_DM = 4.148808e3;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. 4 "round(x) ... rounded to the nearest integer"; ties are not
 * specified by the paper and are read as round-half-up: floor(x + 0.5). */
double orc_round_half_up(double x)
{
    return floor(x + 0.5);
}

/* Eq. 3: Delta T(nu) = (k_DM / dtau) * ((nu0 + nu*dnu)^-2 - nu0^-2), in
 * samples per unit DM.  nu0 is the frequency of channel 0 in MHz, dnu the
 * (signed) channel spacing in MHz, dtau the sampling interval in seconds. */
double orc_partial_delay(double f0_mhz, double df_mhz, double dt_s, int chan)
{
    double f = f0_mhz + (double)chan * df_mhz;
    return (ORC_K_DM / dt_s) * (1.0 / (f * f) - 1.0 / (f0_mhz * f0_mhz));
}

/* Sec. 2.2, time-scrunching.  The "diagonal" DM is where the dispersion
 * curve's gradient on the time-frequency grid reaches one sample per channel
 * everywhere in the band: where the smallest per-channel delay step, between
 * the two highest channels (0 and 1), equals one sample.  This reading (the
 * paper does not say which channel pair) reproduces the paper's projected
 * 1.6x saving on its survey band (Sec. 5.2); see the pins. */
double orc_diagonal_dm(double f0_mhz, double df_mhz, double dt_s)
{
    double step = orc_partial_delay(f0_mhz, df_mhz, dt_s, 1) -
                  orc_partial_delay(f0_mhz, df_mhz, dt_s, 0);
    return step > 0.0 ? 1.0 / step : 0.0;
}

/* Scrunch factor of a trial (Sec. 2.2 and the projection of Sec. 5.2):
 * full resolution below twice the diagonal, then 2 up to 4x the diagonal,
 * 4 up to 8x and so on (at most max_factor). */
int orc_scrunch_factor(double dm, double diag, int max_factor)
{
    int s = 1;
    while (s < max_factor && diag > 0.0 && dm >= 2.0 * (double)s * diag) s *= 2;
    return s;
}

/* Eq. 4 for every (d, c): out[d*nchans + c] = round(DM(d) * Delta T(c)).
 * Returns 0, or -1 on a bad argument (non-positive frequency, negative
 * delay or a delay that does not fit in int32). */
int orc_delay_table(int nchans, double f0_mhz, double df_mhz, double dt_s,
                    const double *dms, int ndm, int32_t *out)
{
    if (nchans <= 0 || ndm < 0 || dt_s <= 0.0 || f0_mhz <= 0.0) return -1;
    if (f0_mhz + (double)(nchans - 1) * df_mhz <= 0.0) return -1;
    for (int d = 0; d < ndm; ++d) {
        for (int c = 0; c < nchans; ++c) {
            double x = dms[d] * orc_partial_delay(f0_mhz, df_mhz, dt_s, c);
            double r = orc_round_half_up(x);
            if (r < 0.0 || r > 2147483647.0) return -1;
            out[(int64_t)d * nchans + c] = (int32_t)r;
        }
    }
    return 0;
}

/* Trial-DM list (Sec. 5.2: 1196 trials for 0 <= DM < 1000 with the HTRU
 * parameters, chosen by bounding the smearing from a wrong trial DM; the
 * rule itself is not printed).  Reading used here, all times in us:
 *   t_s = dtau, w = intrinsic pulse width (40 us in Sec. 5.1),
 *   a   = 2 k_DM |dnu| / nu_c^3   (channel smear per unit DM, nu_c the mean
 *         channel frequency),
 *   b   = a * nchans / 4           (smear across the band of half a DM step),
 *   DM_0 = dm_lo and DM_{i+1} the larger root x of
 *   t_s^2 + w^2 + a^2 x^2 + b^2 (x - DM_i)^2 = tol^2 (t_s^2 + w^2 + a^2 DM_i^2),
 *   keeping trials with DM < dm_hi.
 * Writes at most cap trials; returns the number of trials the rule gives
 * (which may exceed cap), or -1 on a bad argument. */
int orc_dm_list(int nchans, double f0_mhz, double df_mhz, double dt_s,
                double dm_lo, double dm_hi, double width_us, double tol,
                double *out, int cap)
{
    if (nchans <= 0 || dt_s <= 0.0 || tol <= 1.0 || dm_lo < 0.0 || dm_hi <= dm_lo)
        return -1;
    double fc_ghz = (f0_mhz + 0.5 * (double)(nchans - 1) * df_mhz) / 1000.0;
    if (fc_ghz <= 0.0) return -1;
    double a = 2.0 * ORC_K_DM * fabs(df_mhz) / (fc_ghz * fc_ghz * fc_ghz) * 1.0e-3;
    double b = a * (double)nchans / 4.0;
    double ts = dt_s * 1.0e6;
    double base = ts * ts + width_us * width_us;
    int n = 0;
    double dm = dm_lo;
    while (dm < dm_hi) {
        if (n < cap) out[n] = dm;
        ++n;
        if (n > 100000000) return -1;
        double qa = a * a + b * b;
        double qb = -2.0 * b * b * dm;
        double qc = b * b * dm * dm + base - tol * tol * (base + a * a * dm * dm);
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc < 0.0) return -1;
        double next = (-qb + sqrt(disc)) / (2.0 * qa);
        if (!(next > dm)) return -1;
        dm = next;
    }
    return n;
}

/* A[c][t]: one unsigned sample of a packed time-major row (layout above). */
static uint32_t orc_sample(const uint8_t *in, int nbits, int64_t row_stride,
                           int c, int64_t t)
{
    const uint8_t *row = in + t * row_stride;
    if (nbits == 8) return row[c];
    int64_t bit = (int64_t)c * nbits;
    return ((uint32_t)row[bit >> 3] >> (bit & 7)) & ((1u << nbits) - 1u);
}

static int orc_nbits_ok(int nbits)
{
    return nbits == 1 || nbits == 2 || nbits == 4 || nbits == 8;
}

/* Eq. 2 for integer input: D[d][t] = sum_c mask[c] * A[c][t + delay(d,c)],
 * t in [0, nsamps), accumulated exactly in 64 bits.  The input must hold
 * nsamps + max delay rows (the caller guarantees it).  mask may be NULL (all
 * channels kept).  Returns 0, -1 on a bad argument, -2 if a sum does not fit
 * in 32 bits. */
int orc_direct_u32(const uint8_t *in, int nbits, int64_t row_stride, int nchans,
                   int64_t nsamps, const int32_t *delays, int ndm,
                   const uint8_t *mask, uint32_t *out, int64_t out_stride)
{
    if (!orc_nbits_ok(nbits) || nchans <= 0 || nsamps < 0 || ndm < 0) return -1;
    int overflow = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : overflow)
    for (int d = 0; d < ndm; ++d) {
        const int32_t *dl = delays + (int64_t)d * nchans;
        for (int64_t t = 0; t < nsamps; ++t) {
            uint64_t acc = 0;
            for (int c = 0; c < nchans; ++c) {
                uint64_t m = mask ? mask[c] : 1u;
                acc += m * orc_sample(in, nbits, row_stride, c, t + dl[c]);
            }
            if (acc > 0xFFFFFFFFull) overflow = 1;
            out[(int64_t)d * out_stride + t] = (uint32_t)acc;
        }
    }
    return overflow ? -2 : 0;
}

/* Eq. 2 for 32-bit float input (row t = nchans floats at in + t*row_stride
 * elements), accumulated in double.  abssum (may be NULL) receives
 * sum_c |mask[c] * A[c][t + delay(d,c)]|, used to scale float tolerances. */
int orc_direct_f32(const float *in, int64_t row_stride, int nchans, int64_t nsamps,
                   const int32_t *delays, int ndm, const uint8_t *mask,
                   double *out, double *abssum, int64_t out_stride)
{
    if (nchans <= 0 || nsamps < 0 || ndm < 0) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; ++d) {
        const int32_t *dl = delays + (int64_t)d * nchans;
        for (int64_t t = 0; t < nsamps; ++t) {
            double acc = 0.0, aabs = 0.0;
            for (int c = 0; c < nchans; ++c) {
                double m = mask ? (double)mask[c] : 1.0;
                double v = m * (double)in[(t + dl[c]) * row_stride + c];
                acc += v;
                aabs += fabs(v);
            }
            out[(int64_t)d * out_stride + t] = acc;
            if (abssum) abssum[(int64_t)d * out_stride + t] = aabs;
        }
    }
    return 0;
}

/* Eq. 2 at selected points (dsel[i], tsel[i]) only, for checks at sizes
 * where the full transform is too slow on a CPU. */
int orc_direct_points_u32(const uint8_t *in, int nbits, int64_t row_stride,
                          int nchans, const int32_t *delays, const uint8_t *mask,
                          int npts, const int32_t *dsel, const int64_t *tsel,
                          uint32_t *out)
{
    if (!orc_nbits_ok(nbits) || nchans <= 0 || npts < 0) return -1;
    int overflow = 0;
#pragma omp parallel for schedule(static) reduction(| : overflow)
    for (int i = 0; i < npts; ++i) {
        const int32_t *dl = delays + (int64_t)dsel[i] * nchans;
        uint64_t acc = 0;
        for (int c = 0; c < nchans; ++c) {
            uint64_t m = mask ? mask[c] : 1u;
            acc += m * orc_sample(in, nbits, row_stride, c, tsel[i] + dl[c]);
        }
        if (acc > 0xFFFFFFFFull) overflow = 1;
        out[i] = (uint32_t)acc;
    }
    return overflow ? -2 : 0;
}

int orc_direct_points_f32(const float *in, int64_t row_stride, int nchans,
                          const int32_t *delays, const uint8_t *mask, int npts,
                          const int32_t *dsel, const int64_t *tsel, double *out,
                          double *abssum)
{
    if (nchans <= 0 || npts < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < npts; ++i) {
        const int32_t *dl = delays + (int64_t)dsel[i] * nchans;
        double acc = 0.0, aabs = 0.0;
        for (int c = 0; c < nchans; ++c) {
            double m = mask ? (double)mask[c] : 1.0;
            double v = m * (double)in[(tsel[i] + dl[c]) * row_stride + c];
            acc += v;
            aabs += fabs(v);
        }
        out[i] = acc;
        if (abssum) abssum[i] = aabs;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Sub-band dedispersion (Sec. 4.1).  Trials are grouped consecutively,
 * ndm_per_nom per group (the last group may be short); the nominal trial of
 * group g is trial g*ndm_per_nom (the group's lowest DM, i.e. the early edge
 * of App. B).  Sub-band n holds channels [n*N', (n+1)*N').
 *
 * Stage 1: S[g][n][t] = sum_{c' < N'} mask * A[nN'+c'][t + delay(gn, nN'+c')
 *                                                       - delay(gn, nN')],
 *          gn the nominal trial of group g.
 * Stage 2: D[d][t] = sum_{n < N_SB} S[g(d)][n][t + delay(d, nN')].
 * The stage-2 shift is Eq. (eq:combining_subbands): the sum over m < n of the
 * per-sub-band delay increments telescopes to delay(d, nN').  Stage-1 shifts
 * use differences of rounded delays, which keeps the nominal trials exact.
 * ------------------------------------------------------------------------- */

/* Length of the stage-1 rows: nsamps + max_{d,n} delay(d, nN'). */
int64_t orc_subband_len1(const int32_t *delays, int ndm, int nchans,
                         int chans_per_sb, int64_t nsamps)
{
    int nsb = nchans / chans_per_sb;
    int32_t m = 0;
    for (int d = 0; d < ndm; ++d)
        for (int n = 0; n < nsb; ++n) {
            int32_t v = delays[(int64_t)d * nchans + (int64_t)n * chans_per_sb];
            if (v > m) m = v;
        }
    return nsamps + m;
}

/* Nominal trial of group g (trials g*N'_DM .. g*N'_DM + size - 1).  The
 * default is the group's lowest trial, the early-edge alignment App. B
 * analyses; `centred` takes the middle trial instead, which halves the
 * largest DM error between a trial and its nominal DM (App. B, the closing
 * remark on aligning the sub-bands at the centre). */
int orc_subband_nominal(int g, int ndm, int ndm_per_nom, int centred)
{
    int first = g * ndm_per_nom;
    int size = ndm - first < ndm_per_nom ? ndm - first : ndm_per_nom;
    return centred ? first + (size - 1) / 2 : first;
}

/* Input rows needed beyond nsamps: max over d, c of
 * delay(gn(d), c) - delay(gn(d), n0(c)) + delay(d, n0(c)). */
int32_t orc_subband_max_delay(const int32_t *delays, int ndm, int nchans,
                              int chans_per_sb, int ndm_per_nom, int centred)
{
    int32_t m = 0;
    for (int d = 0; d < ndm; ++d) {
        int gn = orc_subband_nominal(d / ndm_per_nom, ndm, ndm_per_nom, centred);
        const int32_t *dn = delays + (int64_t)gn * nchans;
        const int32_t *dd = delays + (int64_t)d * nchans;
        for (int c = 0; c < nchans; ++c) {
            int n0 = (c / chans_per_sb) * chans_per_sb;
            int32_t v = dn[c] - dn[n0] + dd[n0];
            if (v > m) m = v;
        }
    }
    return m;
}

/* Stage 1 into S laid out [ngroups][nsb][len1].  Row (g, n) is computed for
 * t < nsamps + max_{d in g} delay(d, nN') (the part stage 2 reads) and is
 * zero beyond. */
int orc_subband_stage1(const uint8_t *in, int nbits, int64_t row_stride, int nchans,
                       int chans_per_sb, int ndm_per_nom, int centred,
                       const int32_t *delays, int ndm, const uint8_t *mask,
                       int64_t nsamps, int64_t len1, uint32_t *S)
{
    if (!orc_nbits_ok(nbits) || chans_per_sb <= 0 || nchans % chans_per_sb != 0 ||
        ndm_per_nom <= 0 || ndm <= 0)
        return -1;
    int nsb = nchans / chans_per_sb;
    int ngroups = (ndm + ndm_per_nom - 1) / ndm_per_nom;
    int overflow = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(| : overflow)
    for (int g = 0; g < ngroups; ++g) {
        for (int n = 0; n < nsb; ++n) {
            int first = g * ndm_per_nom;
            int dend = first + ndm_per_nom < ndm ? first + ndm_per_nom : ndm;
            int gn = orc_subband_nominal(g, ndm, ndm_per_nom, centred);
            const int32_t *dn = delays + (int64_t)gn * nchans;
            int n0 = n * chans_per_sb;
            int32_t need = 0;
            for (int d = first; d < dend; ++d) {
                int32_t v = delays[(int64_t)d * nchans + n0];
                if (v > need) need = v;
            }
            int64_t tmax = nsamps + need;
            uint32_t *row = S + ((int64_t)g * nsb + n) * len1;
            for (int64_t t = 0; t < len1; ++t) {
                if (t >= tmax) { row[t] = 0; continue; }
                uint64_t acc = 0;
                for (int cp = 0; cp < chans_per_sb; ++cp) {
                    int c = n0 + cp;
                    uint64_t m = mask ? mask[c] : 1u;
                    acc += m * orc_sample(in, nbits, row_stride, c, t + dn[c] - dn[n0]);
                }
                if (acc > 0xFFFFFFFFull) overflow = 1;
                row[t] = (uint32_t)acc;
            }
        }
    }
    return overflow ? -2 : 0;
}

/* Stage 2 from S ([ngroups][nsb][len1]) into D[d][t], t < nsamps. */
int orc_subband_stage2(const uint32_t *S, int nchans, int chans_per_sb,
                       int ndm_per_nom, const int32_t *delays, int ndm,
                       int64_t nsamps, int64_t len1, uint32_t *out,
                       int64_t out_stride)
{
    if (chans_per_sb <= 0 || nchans % chans_per_sb != 0 || ndm_per_nom <= 0) return -1;
    int nsb = nchans / chans_per_sb;
    int overflow = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : overflow)
    for (int d = 0; d < ndm; ++d) {
        int g = d / ndm_per_nom;
        for (int64_t t = 0; t < nsamps; ++t) {
            uint64_t acc = 0;
            for (int n = 0; n < nsb; ++n) {
                int64_t tt = t + delays[(int64_t)d * nchans + (int64_t)n * chans_per_sb];
                acc += S[((int64_t)g * nsb + n) * len1 + tt];
            }
            if (acc > 0xFFFFFFFFull) overflow = 1;
            out[(int64_t)d * out_stride + t] = (uint32_t)acc;
        }
    }
    return overflow ? -2 : 0;
}

/* Appendix B, first form: t_SB <= dDM_nom * [Delta T(N_nu) - Delta T(N_nu - N')]
 * in samples (Delta T of Eq. 3 evaluated at the band edge nu = N_nu), where
 * dDM_nom is the spacing of nominal DMs.  Returns the bound in seconds. */
double orc_subband_smear_bound(double f0_mhz, double df_mhz, double dt_s,
                               int nchans, int chans_per_sb, double dm_nom_step)
{
    double hi = orc_partial_delay(f0_mhz, df_mhz, dt_s, nchans);
    double lo = orc_partial_delay(f0_mhz, df_mhz, dt_s, nchans - chans_per_sb);
    return dm_nom_step * (hi - lo) * dt_s;
}

/* Appendix B, second form (Taylor expansion to first order in N'/N_nu):
 * t_SB ~= dDM_nom * (k_DM / nu0^2) * (-2 (N'/N_nu) lambda / (1+lambda)^3),
 * lambda = dnu * N_nu / nu0.  Seconds. */
double orc_subband_smear_taylor(double f0_mhz, double df_mhz, int nchans,
                                int chans_per_sb, double dm_nom_step)
{
    double lam = df_mhz * (double)nchans / f0_mhz;
    double r = (double)chans_per_sb / (double)nchans;
    return dm_nom_step * (ORC_K_DM / (f0_mhz * f0_mhz)) *
           (-2.0 * r * lam / ((1.0 + lam) * (1.0 + lam) * (1.0 + lam)));
}

/* Eq. (eq:RelativeSmearingSubband): mu_SB = sqrt(W^2 + t_SB^2) / W. */
double orc_relative_smearing(double w_s, double t_sb_s)
{
    return sqrt(w_s * w_s + t_sb_s * t_sb_s) / w_s;
}

/* ---------------------------------------------------------------------------
 * Tree dedispersion (Sec. 3.1) and the piecewise linear tree method
 * (Sec. 3.1.1).
 *
 * The basic tree computes D'[d'][t] = sum_nu A[nu][t + dt'(d', nu)] for the
 * linear trails d' = 0 .. N-1 of a block of N = 2^m channels in m steps:
 *   A^{i+1}[2nu  ][t] = A^i[Phi(i, 2nu)][t] + A^i[Phi(i, 2nu+1)][t + Theta(i, 2nu)]
 *   A^{i+1}[2nu+1][t] = A^i[Phi(i, 2nu)][t] + A^i[Phi(i, 2nu+1)][t + Theta(i, 2nu+1)]
 * with the integer delay Theta of Eq. (tree_integer_delay) and the shuffle
 * Phi of Eq. (shuffle) at radix r = 2^i, all divisions truncated; after the
 * last step row d' holds D'[d'].  The delays it applies are the tree's own
 * approximation of the rounded linear trail of Eq. (tree); they coincide with
 * round(d' nu / (N - 1)) only for small blocks.
 *
 * Each step reads A^i at t + Theta <= t + r, so its output is r samples
 * shorter than its input: from L input samples the tree returns L - (N - 1).
 * ------------------------------------------------------------------------- */

/* Eq. (tree_integer_delay): Theta(i, nu) = [(nu mod 2^{i+1}) + 1] / 2. */
int orc_tree_theta(int i, int nu)
{
    return ((nu % (2 << i)) + 1) / 2;
}

/* Eq. (shuffle): Phi(r, nu) = (nu mod 2) r + nu/2 + (nu/(2r)) r, r = 2^i. */
int orc_tree_phi(int r, int nu)
{
    return (nu % 2) * r + nu / 2 + (nu / (2 * r)) * r;
}

static int orc_is_pow2(int n)
{
    return n > 0 && (n & (n - 1)) == 0;
}

/* The basic tree on n rows (a power of two) of len samples each, a[nu*len +
 * t]; out receives n rows of len - (n - 1) samples, out[d'*(len-n+1) + t].
 * Returns 0, or -1 on a bad argument. */
int orc_tree(const int64_t *a, int n, int64_t len, int64_t *out)
{
    if (!orc_is_pow2(n) || len < n) return -1;
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * (size_t)len);
    int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * (size_t)len);
    if (!cur || !nxt) { free(cur); free(nxt); return -1; }
    memcpy(cur, a, sizeof(int64_t) * (size_t)n * (size_t)len);
    int64_t lcur = len;
    for (int i = 0; (1 << i) < n; ++i) {
        int r = 1 << i;
        int64_t lnext = lcur - r;
        for (int v = 0; v < n / 2; ++v) {
            const int64_t *lo = cur + (int64_t)orc_tree_phi(r, 2 * v) * len;
            const int64_t *hi = cur + (int64_t)orc_tree_phi(r, 2 * v + 1) * len;
            for (int j = 0; j < 2; ++j) {
                int th = orc_tree_theta(i, 2 * v + j);
                int64_t *o = nxt + (int64_t)(2 * v + j) * len;
                for (int64_t t = 0; t < lnext; ++t) o[t] = lo[t] + hi[t + th];
            }
        }
        int64_t *sw = cur; cur = nxt; nxt = sw;
        lcur = lnext;
    }
    for (int d = 0; d < n; ++d)
        memcpy(out + (int64_t)d * lcur, cur + (int64_t)d * len, sizeof(int64_t) * (size_t)lcur);
    free(cur);
    free(nxt);
    return 0;
}

/* Stage-2 quantities of the piecewise linear tree (Sec. 3.1.1) for trial d
 * and sub-band n, from a delay table of nchans + 1 columns (Eq. 4 evaluated
 * at channels 0 .. N_nu, the last one being the band edge nu_{N_s}):
 *   d'_n(d)   = dt(d, nu_{n+1}) - dt(d, nu_n)      (the sub-band's linear DM,
 *               read as the difference of the rounded delays, the first form
 *               the paper prints),
 *   dt''_n(d) = dt(d, nu_n)                        (Eq. combining_subbands:
 *               the sum over m < n of the per-sub-band increments telescopes).
 * Returns -3 if d'_n(d) falls outside 0 .. N'-1 (the trial lies beyond the
 * piecewise diagonal DM of Eq. tree_dm_limit). */
static int orc_tree_stage2_terms(const int32_t *dext, int nchans, int nsub, int d, int n,
                                 int32_t *dprime, int32_t *shift)
{
    const int32_t *row = dext + (int64_t)d * (nchans + 1);
    int32_t a = row[(int64_t)n * nsub], b = row[(int64_t)(n + 1) * nsub];
    *dprime = b - a;
    *shift = a;
    return (*dprime < 0 || *dprime >= nsub) ? -3 : 0;
}

/* Input rows beyond nsamps that the piecewise linear tree reads:
 * max_{d,n} dt''_n(d) + (N' - 1).  -3 as above. */
int64_t orc_tree_max_delay(const int32_t *dext, int ndm, int nchans, int nsub)
{
    int32_t m = 0;
    for (int d = 0; d < ndm; ++d)
        for (int n = 0; n < nchans / nsub; ++n) {
            int32_t dp, sh;
            if (orc_tree_stage2_terms(dext, nchans, nsub, d, n, &dp, &sh)) return -3;
            if (sh > m) m = sh;
        }
    return (int64_t)m + nsub - 1;
}

/* The piecewise linear tree method, integer input.
 * Stage 1 (Eq. subband_result): the basic tree on each sub-band of N' = nsub
 *   channels, S[n][d'][t] = sum_{nu'} A[nu_n + nu'][t + tree delay(d', nu')],
 *   for t < nsamps + max dt''.
 * Stage 2 (Eq. combining_subbands):
 *   D[d][t] = sum_n S[n][d'_n(d)][t + dt''_n(d)].
 * dext is the (ndm) x (nchans + 1) delay table described above.  The input
 * must hold nsamps + orc_tree_max_delay rows.  Returns 0, -1 on a bad
 * argument, -2 if a sum does not fit 32 bits, -3 for a trial beyond the
 * piecewise diagonal DM. */
int orc_tree_piecewise_u32(const uint8_t *in, int nbits, int64_t row_stride, int nchans,
                           int nsub, int64_t nsamps, const int32_t *dext, int ndm,
                           const uint8_t *mask, uint32_t *out, int64_t out_stride)
{
    if (!orc_nbits_ok(nbits) || !orc_is_pow2(nsub) || nchans % nsub != 0 || nsamps <= 0 ||
        ndm <= 0)
        return -1;
    int64_t extra = orc_tree_max_delay(dext, ndm, nchans, nsub);
    if (extra < 0) return (int)extra;
    int nsb = nchans / nsub;
    int64_t len_in = nsamps + extra;             /* input rows read */
    int64_t len1 = len_in - (nsub - 1);          /* stage-1 samples per row */
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)nchans * (size_t)len1);
    if (!S) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int n = 0; n < nsb; ++n) {
        int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)nsub * (size_t)len_in);
        if (!a) { bad = 1; continue; }
        for (int v = 0; v < nsub; ++v) {
            int c = n * nsub + v;
            int64_t m = mask ? mask[c] : 1;
            for (int64_t t = 0; t < len_in; ++t)
                a[(int64_t)v * len_in + t] = m * (int64_t)orc_sample(in, nbits, row_stride, c, t);
        }
        if (orc_tree(a, nsub, len_in, S + (int64_t)n * nsub * len1)) bad = 1;
        free(a);
    }
    if (bad) { free(S); return -1; }
    int overflow = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : overflow)
    for (int d = 0; d < ndm; ++d) {
        for (int64_t t = 0; t < nsamps; ++t) {
            int64_t acc = 0;
            for (int n = 0; n < nsb; ++n) {
                int32_t dp, sh;
                orc_tree_stage2_terms(dext, nchans, nsub, d, n, &dp, &sh);
                acc += S[((int64_t)n * nsub + dp) * len1 + t + sh];
            }
            if (acc < 0 || acc > 0xFFFFFFFFll) overflow = 1;
            out[(int64_t)d * out_stride + t] = (uint32_t)acc;
        }
    }
    free(S);
    return overflow ? -2 : 0;
}

/* Eq. (tree_dm_limit): the piecewise diagonal DM,
 * (N' - 1/2) / (Delta T(N_nu) - Delta T(N_nu - N')). */
double orc_tree_dm_limit(double f0_mhz, double df_mhz, double dt_s, int nchans, int nsub)
{
    double hi = orc_partial_delay(f0_mhz, df_mhz, dt_s, nchans);
    double lo = orc_partial_delay(f0_mhz, df_mhz, dt_s, nchans - nsub);
    return ((double)nsub - 0.5) / (hi - lo);
}

/* Appendix A, Eq. (subband_error): the piecewise linear approximation's
 * smear, t_tree <= (3/4) DM (k_DM / nu0^2) (N'/N_nu)^2 lambda^2 / (1 + lambda)^4,
 * lambda = dnu N_nu / nu0.  Seconds. */
double orc_tree_smear_bound(double dm, double f0_mhz, double df_mhz, int nchans, int nsub)
{
    double lam = df_mhz * (double)nchans / f0_mhz;
    double r = (double)nsub / (double)nchans;
    double q = (1.0 + lam) * (1.0 + lam);
    return 0.75 * dm * (ORC_K_DM / (f0_mhz * f0_mhz)) * r * r * lam * lam / (q * q);
}
