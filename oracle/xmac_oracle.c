/*
 * Plain CPU oracle for the MWA X-engine (cross-multiply and accumulate).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the correlator computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path (the CUDA library) never calls it and shares no code with it.
 *
 * What it computes (the plain definition, no blocking, no reordering):
 *
 *   For every fine channel f and every input pair 0 <= j <= i < N
 *
 *       V[f][i(i+1)/2 + j] += sum_{t < T} x_i(t,f) * conj(x_j(t,f))
 *
 *   i.e. the FX correlator of Eq. 3 (Section 2): the per-channel product of
 *   one input's spectrum with the conjugate of the other's, integrated over
 *   time for the accumulation length (Section 3.4.2, where products are
 *   integrated over a time I), emitted as the packed lower triangle including
 *   the autocorrelations (Appendix C, "GPU Output").  With x = r + i*m:
 *
 *       Re V_ij = sum_t ( r_i r_j + m_i m_j )
 *       Im V_ij = sum_t ( m_i r_j - r_i m_j )
 *
 *   in 64-bit integers.  Section 4.1 states that the GPU correlator was
 *   verified against a simple CPU implementation; this is that comparison
 *   point for the rebuilt X-engine.
 *
 * Input encoding (Appendix A, "Data Format"): each sample is one byte holding
 * a 4-bit two's-complement real part and a 4-bit two's-complement imaginary
 * part ("8-bit (4R+4I)").  Reading taken here: the real part is the high
 * nibble (bits 7..4) and the imaginary part the low nibble (bits 3..0).  The
 * nibble code 8 (value -8) is the paper's "invalid" marker.  By default it is
 * decoded as the value -8; with zero_invalid != 0 a sample in which either
 * nibble is 8 is treated as the complex value 0.
 *
 * Input layout (Appendix C, "GPU Input": time slowest, then channel, then the
 * input index n = 2*station + pol, complex innermost): volt[t][f][n], one byte
 * per complex sample.
 *
 * Output layout: vis[f][i(i+1)/2 + j][2] int64 (re, im), j <= i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 4-bit two's complement: codes 0..7 are 0..7, codes 8..15 are -8..-1. */
static int nibble_value(unsigned code)
{
    code &= 0xFu;
    return code >= 8u ? (int)code - 16 : (int)code;
}

void oracle_decode(const uint8_t *volt, int64_t count, int zero_invalid,
                   int32_t *re, int32_t *im)
{
    for (int64_t k = 0; k < count; ++k) {
        unsigned b = volt[k];
        unsigned hi = (b >> 4) & 0xFu, lo = b & 0xFu;
        if (zero_invalid && (hi == 8u || lo == 8u)) {
            re[k] = 0;
            im[k] = 0;
        } else {
            re[k] = nibble_value(hi);
            im[k] = nibble_value(lo);
        }
    }
}

/* Decode channel f into xr[n*T + t], xi[n*T + t] (a gather, no arithmetic). */
static void gather_channel(const uint8_t *volt, int N, int F, int T, int f,
                           int zero_invalid, int32_t *xr, int32_t *xi)
{
    for (int t = 0; t < T; ++t) {
        const uint8_t *row = volt + ((int64_t)t * F + f) * N;
        for (int n = 0; n < N; ++n) {
            int32_t r, m;
            oracle_decode(row + n, 1, zero_invalid, &r, &m);
            xr[(int64_t)n * T + t] = r;
            xi[(int64_t)n * T + t] = m;
        }
    }
}

/*
 * Packed lower triangle, accumulated into vis (the caller zeroes it for a
 * fresh integration).  Returns 0, or -1 on bad arguments / out of memory.
 */
int oracle_xmac_tri(const uint8_t *volt, int N, int F, int T, int zero_invalid,
                    int64_t *vis)
{
    if (!volt || !vis || N < 1 || F < 1 || T < 0)
        return -1;
    const int64_t P = (int64_t)N * (N + 1) / 2;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int f = 0; f < F; ++f) {
        int32_t *xr = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)(T > 0 ? T : 1));
        int32_t *xi = (int32_t *)malloc(sizeof(int32_t) * (size_t)N * (size_t)(T > 0 ? T : 1));
        if (!xr || !xi) {
            free(xr);
            free(xi);
#pragma omp atomic write
            err = -1;
            continue;
        }
        gather_channel(volt, N, F, T, f, zero_invalid, xr, xi);
        int64_t *vf = vis + (int64_t)f * P * 2;
        for (int i = 0; i < N; ++i) {
            const int32_t *ri = xr + (int64_t)i * T, *mi = xi + (int64_t)i * T;
            for (int j = 0; j <= i; ++j) {
                const int32_t *rj = xr + (int64_t)j * T, *mj = xi + (int64_t)j * T;
                int64_t sre = 0, sim = 0;
                for (int t = 0; t < T; ++t) {
                    sre += (int64_t)ri[t] * rj[t] + (int64_t)mi[t] * mj[t];
                    sim += (int64_t)mi[t] * rj[t] - (int64_t)ri[t] * mj[t];
                }
                int64_t p = (int64_t)i * (i + 1) / 2 + j;
                vf[2 * p] += sre;
                vf[2 * p + 1] += sim;
            }
        }
        free(xr);
        free(xi);
    }
    return err;
}

/* Full N x N matrix vis[f][i][j][2] (both triangles), for symmetry checks. */
int oracle_xmac_full(const uint8_t *volt, int N, int F, int T, int zero_invalid,
                     int64_t *vis)
{
    if (!volt || !vis || N < 1 || F < 1 || T < 0)
        return -1;
    for (int f = 0; f < F; ++f) {
        for (int i = 0; i < N; ++i) {
            for (int j = 0; j < N; ++j) {
                int64_t sre = 0, sim = 0;
                for (int t = 0; t < T; ++t) {
                    const uint8_t *row = volt + ((int64_t)t * F + f) * N;
                    int32_t ri, mi, rj, mj;
                    oracle_decode(row + i, 1, zero_invalid, &ri, &mi);
                    oracle_decode(row + j, 1, zero_invalid, &rj, &mj);
                    sre += (int64_t)ri * rj + (int64_t)mi * mj;
                    sim += (int64_t)mi * rj - (int64_t)ri * mj;
                }
                int64_t p = ((int64_t)f * N + i) * N + j;
                vis[2 * p] = sre;
                vis[2 * p + 1] = sim;
            }
        }
    }
    return 0;
}

/*
 * One visibility V_ij(f) (any i, j; no triangle restriction), for checking
 * sampled outputs of workloads too large to correlate in full on the CPU.
 */
int oracle_xmac_pair(const uint8_t *volt, int N, int F, int T, int zero_invalid,
                     int f, int i, int j, int64_t *out2)
{
    if (!volt || !out2 || f < 0 || f >= F || i < 0 || i >= N || j < 0 || j >= N)
        return -1;
    int64_t sre = 0, sim = 0;
    for (int t = 0; t < T; ++t) {
        const uint8_t *row = volt + ((int64_t)t * F + f) * N;
        int32_t ri, mi, rj, mj;
        oracle_decode(row + i, 1, zero_invalid, &ri, &mi);
        oracle_decode(row + j, 1, zero_invalid, &rj, &mj);
        sre += (int64_t)ri * rj + (int64_t)mi * mj;
        sim += (int64_t)mi * rj - (int64_t)ri * mj;
    }
    out2[0] = sre;
    out2[1] = sim;
    return 0;
}

/*
 * Incoherent beam (Section 3.4: one of the XMAC's other modes): the total
 * power of all inputs, per channel and sample, summed over n_avg consecutive
 * samples:
 *
 *     beam[k][f] = sum_{t = k n_avg}^{(k+1) n_avg - 1}  sum_{n < N} |x_n(t,f)|^2
 *
 * with |x|^2 = r^2 + m^2 of the decoded sample.  out is int64 [T / n_avg][F];
 * T must be a multiple of n_avg.  Returns 0, or -1 on bad arguments.
 */
int oracle_beam(const uint8_t *volt, int N, int F, int T, int n_avg, int zero_invalid,
                int64_t *out)
{
    if (!volt || !out || N < 1 || F < 1 || T < 0 || n_avg < 1 || T % n_avg != 0)
        return -1;
    for (int k = 0; k < T / n_avg; ++k) {
        for (int f = 0; f < F; ++f) {
            int64_t p = 0;
            for (int t = k * n_avg; t < (k + 1) * n_avg; ++t) {
                const uint8_t *row = volt + ((int64_t)t * F + f) * N;
                for (int n = 0; n < N; ++n) {
                    int32_t r, m;
                    oracle_decode(row + n, 1, zero_invalid, &r, &m);
                    p += (int64_t)r * r + (int64_t)m * m;
                }
            }
            out[(int64_t)k * F + f] = p;
        }
    }
    return 0;
}

/*
 * Output remap (Appendix C, "GPU Output"): the X-engine correlates the inputs
 * in the order the PFBs deliver them and emits the lower triangle over those
 * positions; the archived products are per station pair (s1, s2), s2 <= s1,
 * with the 2 x 2 polarisation products inside, in natural input order, and
 * a product the triangle holds only as its conjugate has to be conjugated.
 * Reading taken here: natural input a is station a / 2, polarisation a % 2,
 * and nat_of_pfb[i] is the natural input at PFB position i.
 *
 * Optionally the products are integrated further by f_avg adjacent channels
 * and over n_dumps consecutive dumps ("integrate by a factor of two in each
 * dimension", Section 3.4.3):
 *
 *     out[g][s1(s1+1)/2 + s2][p1][p2] = sum_{d < n_dumps} sum_{f = g f_avg}^{(g+1) f_avg - 1}
 *                                      V^{(d)}_{2 s1 + p1, 2 s2 + p2}(f)
 *
 * where V_AB = tri[i][j] for i = pos(A) >= j = pos(B) and conj(tri[j][i])
 * otherwise.  tri is int64 [n_dumps][F][N(N+1)/2][2] (PFB-order triangles),
 * out int64 [F / f_avg][S(S+1)/2][2][2][2] with S = N / 2.  Returns 0, or -1
 * on bad arguments (odd N, F not a multiple of f_avg, not a permutation).
 */
int oracle_remap(const int64_t *tri, int N, int F, int n_dumps, int f_avg, const int32_t *nat_of_pfb,
                 int64_t *out)
{
    if (!tri || !out || !nat_of_pfb || N < 2 || N % 2 != 0 || F < 1 || n_dumps < 1 || f_avg < 1 ||
        F % f_avg != 0)
        return -1;
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!pos)
        return -1;
    for (int a = 0; a < N; ++a)
        pos[a] = -1;
    for (int i = 0; i < N; ++i) {
        int a = nat_of_pfb[i];
        if (a < 0 || a >= N || pos[a] != -1) {
            free(pos);
            return -1;
        }
        pos[a] = i;
    }
    const int S = N / 2;
    const int64_t P = (int64_t)N * (N + 1) / 2;
    const int64_t Q = (int64_t)S * (S + 1) / 2;
    for (int g = 0; g < F / f_avg; ++g) {
        for (int s1 = 0; s1 < S; ++s1) {
            for (int s2 = 0; s2 <= s1; ++s2) {
                for (int p1 = 0; p1 < 2; ++p1) {
                    for (int p2 = 0; p2 < 2; ++p2) {
                        const int i = pos[2 * s1 + p1], j = pos[2 * s2 + p2];
                        int64_t re = 0, im = 0;
                        for (int d = 0; d < n_dumps; ++d) {
                            for (int f = g * f_avg; f < (g + 1) * f_avg; ++f) {
                                const int64_t *vf = tri + ((int64_t)d * F + f) * P * 2;
                                if (i >= j) {
                                    const int64_t k = (int64_t)i * (i + 1) / 2 + j;
                                    re += vf[2 * k];
                                    im += vf[2 * k + 1];
                                } else {
                                    const int64_t k = (int64_t)j * (j + 1) / 2 + i;
                                    re += vf[2 * k];
                                    im -= vf[2 * k + 1];
                                }
                            }
                        }
                        int64_t *o = out + (((int64_t)g * Q + (int64_t)s1 * (s1 + 1) / 2 + s2) * 4 + p1 * 2 + p2) * 2;
                        o[0] = re;
                        o[1] = im;
                    }
                }
            }
        }
    }
    free(pos);
    return 0;
}

/*
 * Packet ingest (Appendix A "Data Format"; Appendix B): turn one 50 ms bank of
 * PFB packets into the assembled voltage block volt[500][3072][256] (frame,
 * fine channel, input in PFB order).  A packet is 264 bytes: the header word
 * 0x0800, word two and word three with the second tick and the counters, 256
 * sample bytes (four fine channels of 64 PFB inputs), and a 16-bit checksum,
 * the XOR of the 128 data words.  Readings where the appendix is silent:
 * words are most significant byte first; word two holds sec_tick (bit 0),
 * pfb_id (bits 4-5), mgt_id (bits 6-8) and mgt_bank (bits 9-13); word three
 * holds mgt_frame (bits 0-8: values 0-499 need 9 bits), mgt_group (bits
 * 9-10) and mgt_channel (bits 11-15); data byte 64 f2 + k is fine channel
 * 128 mgt_channel + 16 mgt_id + 4 mgt_group + f2, input 64 pfb_id + k.
 *
 * A packet is rejected (counted, not written) if its header is not 0x0800,
 * its checksum does not match, or a field is out of range for this bank
 * (mgt_bank != bank, mgt_channel >= 24, mgt_frame >= 500, or sec_tick set on
 * a packet that is not the second's first).  Every (frame, group of four
 * channels, PFB) slot that no good packet filled is written with the byte
 * 0x88 (both parts code 8, the appendix's invalid marker).  counters:
 * [0] good, [1] bad header, [2] bad checksum, [3] bad field, [4] duplicate
 * (a slot filled again; the later packet's bytes stay), [5] missing slots.
 */
#define PKT_FRAMES 500
#define PKT_CHANNELS 3072
#define PKT_INPUTS 256
#define PKT_GROUPS (PKT_CHANNELS / 4)

int oracle_ingest(const uint8_t *pk, int64_t n_packets, int bank, uint8_t *volt, int64_t *counters)
{
    if ((!pk && n_packets > 0) || n_packets < 0 || !volt || !counters || bank < 0 || bank > 31)
        return -1;
    const int64_t n_slots = (int64_t)PKT_FRAMES * PKT_GROUPS * 4;
    uint8_t *seen = (uint8_t *)calloc((size_t)n_slots, 1);
    if (!seen)
        return -1;
    for (int c = 0; c < 6; ++c)
        counters[c] = 0;
    for (int64_t q = 0; q < n_packets; ++q) {
        const uint8_t *b = pk + q * 264;
        const unsigned header = ((unsigned)b[0] << 8) | b[1];
        if (header != 0x0800u) {
            counters[1]++;
            continue;
        }
        unsigned xhi = 0, xlo = 0;
        for (int w = 0; w < 128; ++w) {
            xhi ^= b[6 + 2 * w];
            xlo ^= b[7 + 2 * w];
        }
        if (xhi != b[262] || xlo != b[263]) {
            counters[2]++;
            continue;
        }
        const unsigned w2 = ((unsigned)b[2] << 8) | b[3];
        const unsigned w3 = ((unsigned)b[4] << 8) | b[5];
        const int tick = (int)(w2 & 1u);
        const int pfb = (int)((w2 >> 4) & 3u);
        const int mgt = (int)((w2 >> 6) & 7u);
        const int bnk = (int)((w2 >> 9) & 31u);
        const int frame = (int)(w3 & 511u);
        const int grp = (int)((w3 >> 9) & 3u);
        const int chan = (int)((w3 >> 11) & 31u);
        const int first = bnk == 0 && chan == 0 && grp == 0 && frame == 0;
        if (bnk != bank || chan >= 24 || frame >= PKT_FRAMES || (tick && !first)) {
            counters[3]++;
            continue;
        }
        const int cgroup = 32 * chan + 4 * mgt + grp;          /* fine channel / 4 */
        const int64_t slot = ((int64_t)frame * PKT_GROUPS + cgroup) * 4 + pfb;
        if (seen[slot])
            counters[4]++;
        seen[slot] = 1;
        counters[0]++;
        for (int f2 = 0; f2 < 4; ++f2) {
            const int f = 4 * cgroup + f2;
            for (int k = 0; k < 64; ++k)
                volt[((int64_t)frame * PKT_CHANNELS + f) * PKT_INPUTS + 64 * pfb + k] = b[6 + 64 * f2 + k];
        }
    }
    for (int frame = 0; frame < PKT_FRAMES; ++frame) {
        for (int cgroup = 0; cgroup < PKT_GROUPS; ++cgroup) {
            for (int pfb = 0; pfb < 4; ++pfb) {
                if (seen[((int64_t)frame * PKT_GROUPS + cgroup) * 4 + pfb])
                    continue;
                counters[5]++;
                for (int f2 = 0; f2 < 4; ++f2)
                    for (int k = 0; k < 64; ++k)
                        volt[((int64_t)frame * PKT_CHANNELS + 4 * cgroup + f2) * PKT_INPUTS + 64 * pfb + k] = 0x88;
            }
        }
    }
    free(seen);
    return 0;
}

/*
 * Fine polyphase filterbank, the second channeliser of the F stage (Section
 * 3.2.1): a critically sampled, n_taps-tap, 128-point filter-response-weighted
 * DFT that splits each 1.28 MHz coarse channel into 128 fine channels of
 * 10 kHz (one output sample per 128 input samples).  The paper gives the
 * structure (12 taps, 128 points) but not the window coefficients, so the
 * window h[p * 128 + n] (p < n_taps, n < 128) is an input.
 *
 * For coarse channel q, input i and frame m:
 *
 *     u_m[n] = sum_{p < n_taps} h[p * 128 + n] * x_qi[(m + p) * 128 + n]     (n < 128)
 *     Y_m[k] = sum_{n < 128} u_m[n] * exp(-2 pi i k n / 128)                 (k < 128)
 *
 * Readings taken here: frame m spans the input samples [128 m, 128 (m + n_taps)),
 * and tap p weights the p-th block of 128 samples of that span (for the usual
 * symmetric prototype filter this is the same as the convolution form); the
 * DFT is the forward one (negative exponent); fine channel c = (k + 64) mod 128,
 * so that c = 0 is the lowest frequency of the coarse channel and c = 64 its
 * centre (the usual order of a channelised band).
 *
 * x is int8 [Q][N][S][2] (real, imaginary), S a multiple of 128 and at least
 * 128 n_taps; M = S / 128 - n_taps + 1 frames.  Output channel q * 128 + c:
 *   spec  double [M][Q * 128][N][2]  Y_m[k] (may be NULL);
 *   volt  uint8  [M][Q * 128][N]     the 4+4-bit sample of Appendix A
 *         (real part in the high nibble) of clamp(rint(scale * Y), -7, 7) per
 *         component, rounding half to even; the X-engine's input layout, so the
 *         two stages chain (may be NULL).
 * Returns 0, or -1 on bad arguments.
 */
static int fpfb_q4(double v)
{
    double r = rint(v);
    if (r > 7.0)
        r = 7.0;
    if (r < -7.0)
        r = -7.0;
    return (int)r;
}

int oracle_fine_pfb(const int8_t *x, int Q, int N, int64_t S, const double *h, int n_taps,
                    double scale, double *spec, uint8_t *volt)
{
    const int L = 128;
    if (!x || !h || Q < 1 || N < 1 || n_taps < 1 || S % L != 0 || S < (int64_t)L * n_taps)
        return -1;
    const int64_t M = S / L - n_taps + 1;
    const int64_t C = (int64_t)Q * L;
    const double two_pi = 6.283185307179586476925286766559;
    double cs[128], sn[128];
    for (int r = 0; r < L; ++r) {
        cs[r] = cos(two_pi * r / L);
        sn[r] = sin(two_pi * r / L);
    }
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int q = 0; q < Q; ++q) {
        for (int i = 0; i < N; ++i) {
            const int8_t *xi = x + ((int64_t)q * N + i) * S * 2;
            double ur[128], um[128];
            for (int64_t m = 0; m < M; ++m) {
                for (int n = 0; n < L; ++n) {
                    double ar = 0.0, am = 0.0;
                    for (int p = 0; p < n_taps; ++p) {
                        const int64_t s = (m + p) * L + n;
                        ar += h[p * L + n] * xi[2 * s];
                        am += h[p * L + n] * xi[2 * s + 1];
                    }
                    ur[n] = ar;
                    um[n] = am;
                }
                for (int k = 0; k < L; ++k) {
                    double yr = 0.0, ym = 0.0;
                    for (int n = 0; n < L; ++n) {
                        /* exp(-2 pi i k n / L) = cos - i sin */
                        const int r = (k * n) % L;
                        yr += ur[n] * cs[r] + um[n] * sn[r];
                        ym += um[n] * cs[r] - ur[n] * sn[r];
                    }
                    const int c = (k + L / 2) % L;
                    const int64_t o = (m * C + (int64_t)q * L + c) * N + i;
                    if (spec) {
                        spec[2 * o] = yr;
                        spec[2 * o + 1] = ym;
                    }
                    if (volt)
                        volt[o] = (uint8_t)(((fpfb_q4(scale * yr) & 15) << 4) | (fpfb_q4(scale * ym) & 15));
                }
            }
        }
    }
    return 0;
}

/* Set the number of OpenMP threads of the triangle routine (n >= 1); returns
 * the number in effect afterwards. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Number of OpenMP threads the triangle routine would use (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
