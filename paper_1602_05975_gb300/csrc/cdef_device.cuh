// Device-side building blocks of the CDEF hot path (arXiv 1602.05975):
// the per-8x8 direction search (section 2, Algorithm 1), the per-block
// parameter derivation (section 3.2, eq. 13) and the constraint of eq. 7.
// Integer arithmetic throughout; results are bit-exact by construction.
#pragma once

#include <cstdint>

namespace cdefgb {

// Section 2, Fig. 1 (figure missing; reading): line number of pixel (row i,
// column j) of an 8x8 block for direction d.  d = 0 is the 45-degree
// up-right diagonal, each next d turns clockwise by about 22.5 degrees,
// d + 4 is perpendicular to d.
__host__ __device__ constexpr int line_of(int d, int i, int j)
{
    return d == 0 ? i + j
         : d == 1 ? i + (j >> 1)
         : d == 2 ? i
         : d == 3 ? 3 + i - (j >> 1)
         : d == 4 ? 7 + i - j
         : d == 5 ? 3 - (i >> 1) + j
         : d == 6 ? j
         : (i >> 1) + j;
}

// 840 / N_{d,k}: the cardinality of each line is at most 8 and divides the
// least common multiple 840 (section 2), so every weight is an integer.
struct LineWeights {
    int w[8][15];
};

__host__ __device__ constexpr LineWeights make_line_weights()
{
    LineWeights t{};
    int cnt[8][15] = {};
    for (int d = 0; d < 8; d++)
        for (int i = 0; i < 8; i++)
            for (int j = 0; j < 8; j++)
                cnt[d][line_of(d, i, j)]++;
    for (int d = 0; d < 8; d++)
        for (int k = 0; k < 15; k++)
            t.w[d][k] = cnt[d][k] ? 840 / cnt[d][k] : 0;
    return t;
}

// Primary tap offsets (row, column) at distance 1 and 2 along d (Fig. 3,
// figure missing; reading: the next pixels on the filtered pixel's line of
// Fig. 1).  Each is used with both signs:
//   d:     0       1       2       3       4       5       6       7
//   k=0 (-1, 1) ( 0, 1) ( 0, 1) ( 0, 1) ( 1, 1) ( 1, 0) ( 1, 0) ( 1, 0)
//   k=1 (-2, 2) (-1, 2) ( 0, 2) ( 1, 2) ( 2, 2) ( 2, 1) ( 2, 0) ( 2,-1)
__host__ __device__ constexpr int tap_dr(int d, int k)
{
    return k == 0 ? (d == 0 ? -1 : (d == 4 || d >= 5) ? 1 : 0)
                  : (d == 0 ? -2 : d == 1 ? -1 : d == 2 ? 0 : d == 3 ? 1 : 2);
}
__host__ __device__ constexpr int tap_dc(int d, int k)
{
    return k == 0 ? (d <= 4 ? 1 : 0)
                  : (d <= 4 ? 2 : d == 5 ? 1 : d == 6 ? 0 : -1);
}

__device__ __forceinline__ int ilog2(int s) { return 31 - __clz(s); }

// Eq. 13 (reading for 2^10 <= v < 2^16: the log term counts as 0).
__device__ __forceinline__ int adjust_strength(int pri, int v)
{
    if (v < 1024) return 0;
    const int q = v >> 16;
    const int i = q ? min(ilog2(q), 12) : 0;
    return (pri * (4 + i) + 8) >> 4;
}

// Effective per-8x8 parameters of one plane (section 3.2): strengths after
// the contrast adjustment (luma) and the bit-depth scaling, the shift
// D - floor(log2 S) of eq. 7 for each tap set (the damping is chroma D - 1,
// raised to floor(log2 S_p); the bit-depth offset of D cancels against the
// scaled log2), and the primary weights picked by the parity of the
// unscaled strength (Fig. 3 caption: even 4/2, odd 3/3 in sixteenths).
struct Eff {
    int pri, sec;    // scaled strengths
    int psh, ssh;    // eq. 7 shifts
    int w0, w1;      // primary near / far weights
};

__device__ __forceinline__ Eff make_eff(int pri_raw, int sec_raw, int damping,
                                        bool chroma, int v, int sh8)
{
    const int pri = chroma ? pri_raw : adjust_strength(pri_raw, v);
    int D = chroma ? damping - 1 : damping;
    const int lp = pri ? ilog2(pri) : 0;
    if (pri && D < lp) D = lp;
    Eff e;
    e.w0 = (pri & 1) ? 3 : 4;
    e.w1 = (pri & 1) ? 3 : 2;
    e.pri = pri << sh8;
    e.sec = sec_raw << sh8;
    e.psh = pri ? D - lp : 0;
    e.ssh = sec_raw ? max(0, D - ilog2(sec_raw)) : 0;
    return e;
}

// Eq. 7 with the anti-symmetric reading of its d < 0 branch:
// sign(d) * min(|d|, max(0, S - (|d| >> shift))).  S = 0 gives 0.
__device__ __forceinline__ int constrain(int diff, int S, int shift)
{
    const int a = abs(diff);
    const int m = min(a, max(0, S - (a >> shift)));
    return diff < 0 ? -m : m;
}

// Eq. 8 rounding of sum/16, ties away from zero.
__device__ __forceinline__ int round16(int sum)
{
    return (sum + 8 - (sum < 0)) >> 4;
}

// Algorithm 1 on one 8x8 block.  `px(i, j)` returns the raw sample; sh8
// brings it to 8 bits (section 2), then it is centred by -128.  Line sums
// are accumulated row by row; the pairs of horizontally adjacent pixels
// feed directions 1 and 3 together, as do pairs of rows for 5 and 7.
// Returns the direction; *var receives s_best - s_{(best+4) mod 8}.
template <typename PX>
__device__ __forceinline__ int find_dir_8x8(PX px, int sh8, int *var)
{
    constexpr LineWeights LW = make_line_weights();
    int part[8][15];
#pragma unroll
    for (int d = 0; d < 8; d++)
#pragma unroll
        for (int k = 0; k < 15; k++) part[d][k] = 0;

#pragma unroll
    for (int i = 0; i < 8; i++) {
        int x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = (px(i, j) >> sh8) - 128;
        int pairs[4];
#pragma unroll
        for (int m = 0; m < 4; m++) pairs[m] = x[2 * m] + x[2 * m + 1];
        int row = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            row += x[j];
            part[0][line_of(0, i, j)] += x[j];
            part[4][line_of(4, i, j)] += x[j];
            part[5][line_of(5, i, j)] += x[j];
            part[6][line_of(6, i, j)] += x[j];
            part[7][line_of(7, i, j)] += x[j];
        }
        part[2][i] += row;
#pragma unroll
        for (int m = 0; m < 4; m++) {
            part[1][line_of(1, i, 2 * m)] += pairs[m];
            part[3][line_of(3, i, 2 * m)] += pairs[m];
        }
    }

    int cost[8];
#pragma unroll
    for (int d = 0; d < 8; d++) {
        int s = 0;
#pragma unroll
        for (int k = 0; k < 15; k++)
            if (LW.w[d][k]) s += part[d][k] * part[d][k] * LW.w[d][k];
        cost[d] = s;
    }
    int best = 0, best_cost = cost[0];
#pragma unroll
    for (int d = 1; d < 8; d++)
        if (cost[d] > best_cost) { best_cost = cost[d]; best = d; }
    int opp = 0;
#pragma unroll
    for (int d = 0; d < 8; d++)
        if (d == ((best + 4) & 7)) opp = cost[d];
    *var = best_cost - opp;
    return best;
}

}  // namespace cdefgb
