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

/* Number of OpenMP threads the triangle routine would use (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
