// Checkpoint files of a chain state (host side): the header format, its
// checks and the payload checksum.  The long runs of Sec. IV (more than 1e5
// periods) are resumable from such a file; sv_save / sv_load (sv_api.cu)
// stream the amplitudes through these helpers.
//
// Layout, little-endian:
//   bytes  0..7   magic "FLQSVCK1"
//   bytes  8..11  int32  L
//   bytes 12..15  int32  precision (SV_C64, SV_C128 or SV_DF64)
//   bytes 16..23  int64  period counter
//   bytes 24..31  uint64 payload bytes (8 or 16 bytes x 2^L)
//                 (SV_DF64: the double-float words as held on the device)
//   bytes 32..39  uint64 checksum of the payload
//   bytes 40..47  uint64 checksum of bytes 0..39
//   bytes 48..    the amplitudes, natural layout (site i = bit i), (re, im)
// Checksum: FNV-1a (64-bit offset basis and prime) over the data taken as
// little-endian 64-bit words.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sv_internal.h"

namespace fsv {

namespace {
constexpr char kMagic[8] = {'F', 'L', 'Q', 'S', 'V', 'C', 'K', '1'};
constexpr uint64_t kFnvBasis = 14695981039346656037ull;
constexpr uint64_t kFnvPrime = 1099511628211ull;

uint64_t load_le64(const unsigned char* p) {
  uint64_t v = 0;
  for (int b = 7; b >= 0; --b) v = (v << 8) | p[b];
  return v;
}
void store_le64(unsigned char* p, uint64_t v) {
  for (int b = 0; b < 8; ++b) p[b] = (unsigned char)(v >> (8 * b));
}
}  // namespace

uint64_t ckpt_sum_begin() { return kFnvBasis; }

uint64_t ckpt_sum_update(uint64_t h, const void* data, size_t bytes) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t k = 0; k + 8 <= bytes; k += 8) {
    h ^= load_le64(p + k);
    h *= kFnvPrime;
  }
  return h;
}

void ckpt_encode_header(const CkptHeader& h, unsigned char out[kCkptHeaderBytes]) {
  std::memset(out, 0, kCkptHeaderBytes);
  std::memcpy(out, kMagic, 8);
  store_le64(out + 8, (uint64_t)(uint32_t)h.L | ((uint64_t)(uint32_t)h.precision << 32));
  store_le64(out + 16, (uint64_t)h.period);
  store_le64(out + 24, h.payload_bytes);
  store_le64(out + 32, h.payload_sum);
  store_le64(out + 40, ckpt_sum_update(ckpt_sum_begin(), out, 40));
}

bool ckpt_decode_header(const unsigned char in[kCkptHeaderBytes], CkptHeader* h) {
  if (std::memcmp(in, kMagic, 8) != 0) return false;
  if (load_le64(in + 40) != ckpt_sum_update(ckpt_sum_begin(), in, 40)) return false;
  const uint64_t lp = load_le64(in + 8);
  h->L = (int)(int32_t)(uint32_t)(lp & 0xffffffffu);
  h->precision = (int)(int32_t)(uint32_t)(lp >> 32);
  h->period = (int64_t)load_le64(in + 16);
  h->payload_bytes = load_le64(in + 24);
  h->payload_sum = load_le64(in + 32);
  if (h->L < 2 || h->L > 34) return false;
  if (h->precision != SV_C64 && h->precision != SV_C128 && h->precision != SV_DF64) return false;
  if (h->precision != SV_C64 && h->L > 33) return false;
  if (h->period < 0) return false;
  const uint64_t amp = h->precision == SV_C64 ? 8 : 16;
  return h->payload_bytes == (amp << h->L);
}

}  // namespace fsv

extern "C" int sv_checkpoint_info(const char* path, int* L, int* precision, int64_t* period) {
  if (!path) return SV_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return SV_EINVAL;
  unsigned char hb[fsv::kCkptHeaderBytes];
  fsv::CkptHeader h;
  int rc = SV_OK;
  if (std::fread(hb, 1, sizeof(hb), f) != sizeof(hb) || !fsv::ckpt_decode_header(hb, &h)) {
    rc = SV_EINVAL;
  } else {
    std::vector<unsigned char> buf((size_t)1 << 24);
    uint64_t sum = fsv::ckpt_sum_begin(), left = h.payload_bytes;
    while (left > 0 && rc == SV_OK) {
      const size_t want = (size_t)std::min<uint64_t>(left, buf.size());
      if (std::fread(buf.data(), 1, want, f) != want) rc = SV_EINVAL;
      else sum = fsv::ckpt_sum_update(sum, buf.data(), want);
      left -= want;
    }
    if (rc == SV_OK && (sum != h.payload_sum || std::fgetc(f) != EOF)) rc = SV_EINVAL;
  }
  std::fclose(f);
  if (rc == SV_OK) {
    if (L) *L = h.L;
    if (precision) *precision = h.precision;
    if (period) *period = h.period;
  }
  return rc;
}
