// Internal declarations shared by the host builder (builder.cpp) and the device
// runtime (device.cu) of libpb.so.  Not part of the public ABI (include/pb.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pb.h"

namespace pb {

constexpr double kHbar = 0.6582119569;  // eV fs
constexpr double kBoltz = 8.617333262e-5;  // eV / K
constexpr double kPi = 3.14159265358979323846;

// Partner index and phonon branch packed in one 32-bit word: bits [0,24) partner window
// index, bits [24,32) branch.  Limits nstate to 2^24 and nmodes to 255.
constexpr uint32_t kPartnerBits = 24;
constexpr uint32_t kPartnerMask = (1u << kPartnerBits) - 1u;
constexpr int64_t kMaxStates = (int64_t)1 << kPartnerBits;

// Rows are padded to a multiple of this many channels on the device so that every row
// (and every work item) starts on a 16-byte boundary for all per-channel arrays.
constexpr int kRowPad = 8;

int set_error(int code, const char *fmt, ...);
void clear_error();

}  // namespace pb

// Host CSR built by pb_build_channels (rows = window states in ascending full-grid id).
struct pb_channels {
  int32_t nk[3] = {0, 0, 0};
  int32_t nbands = 0, nmodes = 0;
  int64_t nstate = 0, nch = 0, nq = 0, max_row = 0;
  double T = 0.0, sigma = 0.0;
  std::vector<int32_t> state_ids;  // [nstate] full-grid id
  std::vector<int32_t> kidx;       // [nstate] k-point index ik of each window state
  std::vector<double> eps;         // [nstate] band energy
  std::vector<double> vel;         // [nstate][3] (empty if the model had none)
  std::vector<double> omega;       // [nq][nmodes]
  std::vector<int64_t> row_ptr;    // [nstate+1]
  std::vector<int32_t> col;        // [nch] partner window index
  std::vector<uint8_t> nu;         // [nch] branch
  std::vector<double> g2;          // [nch] |g|^2, eV^2
  bool closed = false;             // the builder verified that every channel's reverse exists with equal |g|^2
};
