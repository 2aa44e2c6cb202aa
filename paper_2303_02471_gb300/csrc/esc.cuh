// ESC accumulator of the light columns (Section 4): shapes and launcher.
#pragma once

#include "kernels.cuh"

namespace spg {

constexpr int kEscWarps = 8;       // warps per CTA, each working its own tiles
constexpr int kEscTile = 256;      // products one warp tile holds
constexpr int kEscRadixBits = 8;   // digit width of the radix sort
// Bins whose largest Op_j is at most this sort by counting within columns
// (see k_esc) instead of the radix sort.
constexpr int kEscRankOpMax = 64;
// How a tile is sorted: radix passes; ranks counted over an aligned window
// around the column (composite keys of column, row and position fit 32
// bits); ranks counted over the column alone (row and position fit).
constexpr int kEscRadix = 0;
constexpr int kEscRankWindow = 1;
constexpr int kEscRankExact = 2;

// Tile shape of one lane-group bin: columns per tile, row bits of the keys,
// radix passes over the key bits (none when ranked) and the sort's form.
struct EscShape {
    int ct = 0;
    int rb = 0;
    int passes = 0;
    int rank = kEscRadix;
};

// Shape of bin `bin` for a product whose forward passes number m rows; false
// when the bin is no lane-group bin or the keys do not fit 32 bits.
bool esc_shape(int bin, int64_t m, EscShape &e);

// values = false: run counts into cnt_out[j + 1] (symbolic).  values = true:
// C's rows and values at base[j] + rank; the counts are written to cnt_out
// when given (single pass), else checked against base[j + 1] - base[j].
cudaError_t launch_esc_bin(const BinTask &t, const Operands &o, const int64_t *base, int64_t *cnt_out,
                           int32_t *Crow, void *Cval, bool values, int dtype, const EscShape &e, int sms,
                           cudaStream_t s);

}  // namespace spg
