// The Markov chain of HMC trajectories with the heatbath and the Metropolis
// uniform drawn on the device (Sec. I), dH spikes marked (Sec. III), and
// checkpoints of the gauge field with a CRC-32 of the links.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "hmc_host.h"

using namespace hmc;

namespace {

constexpr size_t kHeaderBytes = 80;
const char kMagic[8] = {'H', 'M', 'C', 'C', 'K', 'P', 'T', '1'};

// CRC-32 with the reflected IEEE 802.3 polynomial 0xEDB88320, initial value
// and final xor all ones (the checksum of zlib, PNG and Ethernet)
struct Crc32 {
  uint32_t table[256];
  Crc32() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
  }
  uint32_t update(uint32_t crc, const unsigned char *p, size_t n) const {
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
  }
};

const Crc32 &crc_table() {
  static const Crc32 t;
  return t;
}

bool little_endian() {
  const uint32_t one = 1;
  unsigned char b;
  memcpy(&b, &one, 1);
  return b == 1;
}

void put(unsigned char *h, size_t off, const void *v, size_t n) { memcpy(h + off, v, n); }
void get(const unsigned char *h, size_t off, void *v, size_t n) { memcpy(v, h + off, n); }

}  // namespace

extern "C" {

int hmc_chain(hmc_ctx *ctx, const hmc_lattice *lat, void *U, const hmc_traj_params *prm,
              const hmc_chain_params *cp, hmc_traj_result *results) {
  if (!ctx) return HMC_EINVAL;
  TRY(check_lattice(ctx, lat));
  if (!U || !prm || !cp || !results || cp->n_traj < 0)
    return fail(ctx, HMC_EINVAL, "chain: bad arguments");
  TRY(check_aligned(ctx, "chain", {U}));
  const Geo g = make_geo(*lat);
  TRY(traj_check(ctx, g, prm));
  const int nf = traj_eta_fields(prm);
  const size_t ab = (size_t)g.Vh * 2 * 4 * 8 * sizeof(double);
  double *P = (double *)workspace(ctx, "ch_p", ab);
  void *eta = workspace(ctx, "ch_eta", spinor_bytes(g, HMC_F64, 1) * nf);
  double *u = (double *)workspace(ctx, "ch_u", sizeof(double));
  if (!P || !eta || !u) return HMC_ENOMEM;
  for (int t = 0; t < cp->n_traj; ++t) {
    const uint64_t c = cp->counter0 + (uint64_t)t;
    TRY(random_momenta(ctx, g, P, cp->seed, c));
    TRY(random_sources(ctx, g, eta, nf, cp->seed, c));
    TRY(random_uniforms(ctx, u, 1, cp->seed, HMC_STREAM_METROPOLIS, c));
    double uh = 0.0;
    TRY(cuda_ok(ctx, cudaMemcpyAsync(&uh, u, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                "chain: Metropolis uniform"));
    TRY(host_sync(ctx, "chain: Metropolis uniform"));
    TRY(hmc_trajectory(ctx, lat, U, prm, P, eta, uh, &results[t], nullptr, nullptr));
    results[t].spike =
        cp->spike_threshold > 0.0 && std::fabs(results[t].dH) > cp->spike_threshold ? 1 : 0;
  }
  return HMC_OK;
}

int hmc_checkpoint_write(hmc_ctx *ctx, const char *path, const hmc_checkpoint_info *info,
                         const double *U_canon) {
  if (!path || !info || !U_canon) return fail(ctx, HMC_EINVAL, "checkpoint: NULL argument");
  if (!little_endian()) return fail(ctx, HMC_EINVAL, "checkpoint: big-endian host");
  size_t V = 1;
  for (int d = 0; d < 4; ++d) {
    if (info->L[d] < 1) return fail(ctx, HMC_EINVAL, "checkpoint: bad extent %d", info->L[d]);
    V *= (size_t)info->L[d];
  }
  const size_t nbytes = V * 72 * sizeof(double);
  unsigned char h[kHeaderBytes] = {0};
  put(h, 0, kMagic, 8);
  for (int d = 0; d < 4; ++d) {
    const int32_t l = info->L[d];
    put(h, 8 + 4 * d, &l, 4);
  }
  put(h, 24, &info->beta, 8);
  put(h, 32, &info->kappa, 8);
  put(h, 40, &info->seed, 8);
  put(h, 48, &info->trajectory, 8);
  put(h, 56, &info->rng_counter, 8);
  put(h, 64, &info->plaquette, 8);
  const uint32_t crc = crc_table().update(0, (const unsigned char *)U_canon, nbytes);
  put(h, 72, &crc, 4);
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(ctx, HMC_EINVAL, "checkpoint: cannot open %s", tmp.c_str());
  const bool ok = fwrite(h, 1, kHeaderBytes, f) == kHeaderBytes &&
                  fwrite(U_canon, 1, nbytes, f) == nbytes;
  if (fclose(f) != 0 || !ok) {
    remove(tmp.c_str());
    return fail(ctx, HMC_EINVAL, "checkpoint: write to %s failed", tmp.c_str());
  }
  if (rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return fail(ctx, HMC_EINVAL, "checkpoint: cannot rename to %s", path);
  }
  return HMC_OK;
}

int hmc_checkpoint_read(hmc_ctx *ctx, const char *path, hmc_checkpoint_info *info,
                        double *U_canon, size_t n_doubles) {
  if (!path || !info) return fail(ctx, HMC_EINVAL, "checkpoint: NULL argument");
  if (!little_endian()) return fail(ctx, HMC_EINVAL, "checkpoint: big-endian host");
  FILE *f = fopen(path, "rb");
  if (!f) return fail(ctx, HMC_EINVAL, "checkpoint: cannot open %s", path);
  unsigned char h[kHeaderBytes];
  if (fread(h, 1, kHeaderBytes, f) != kHeaderBytes || memcmp(h, kMagic, 8) != 0) {
    fclose(f);
    return fail(ctx, HMC_EINVAL, "checkpoint: %s is not a checkpoint", path);
  }
  hmc_checkpoint_info in{};
  size_t V = 1;
  for (int d = 0; d < 4; ++d) {
    int32_t l;
    get(h, 8 + 4 * d, &l, 4);
    in.L[d] = l;
    if (l < 1) {
      fclose(f);
      return fail(ctx, HMC_EINVAL, "checkpoint: bad extent %d", l);
    }
    V *= (size_t)l;
  }
  get(h, 24, &in.beta, 8);
  get(h, 32, &in.kappa, 8);
  get(h, 40, &in.seed, 8);
  get(h, 48, &in.trajectory, 8);
  get(h, 56, &in.rng_counter, 8);
  get(h, 64, &in.plaquette, 8);
  uint32_t crc_file;
  get(h, 72, &crc_file, 4);
  const size_t nbytes = V * 72 * sizeof(double);
  if (U_canon && n_doubles != V * 72) {
    fclose(f);
    return fail(ctx, HMC_EINVAL, "checkpoint: buffer of %zu doubles, file holds %zu", n_doubles,
                V * 72);
  }
  // the CRC is checked whether or not the links are wanted
  uint32_t crc = 0;
  size_t done = 0;
  unsigned char chunk[1 << 16];
  while (done < nbytes) {
    const size_t want = nbytes - done < sizeof(chunk) ? nbytes - done : sizeof(chunk);
    unsigned char *dst = U_canon ? (unsigned char *)U_canon + done : chunk;
    if (fread(dst, 1, want, f) != want) {
      fclose(f);
      return fail(ctx, HMC_EINVAL, "checkpoint: %s is truncated", path);
    }
    crc = crc_table().update(crc, dst, want);
    done += want;
  }
  fclose(f);
  if (crc != crc_file)
    return fail(ctx, HMC_EINVAL, "checkpoint: CRC mismatch in %s (%08x, stored %08x)", path, crc,
                crc_file);
  *info = in;
  return HMC_OK;
}

}  // extern "C"
