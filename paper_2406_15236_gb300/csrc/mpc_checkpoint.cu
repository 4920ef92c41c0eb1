// Checkpoint files (Sec. III.G.2, "Input/Output"): parameters in a text file, particle
// data ordered by unshifted cell and per-cell counts and offsets in binary files.  Host
// code only; the state goes through mpc_get_state / mpc_set_state.
#include <algorithm>
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "mpc.h"
#include "mpc_host.h"

using namespace mpc::host;

namespace {

constexpr int kFormat = 1;

bool little_endian() {
  const uint32_t one = 1;
  unsigned char b;
  std::memcpy(&b, &one, 1);
  return b == 1;
}

struct File {
  FILE* f = nullptr;
  explicit File(const std::string& path, const char* mode) : f(std::fopen(path.c_str(), mode)) {}
  ~File() {
    if (f) std::fclose(f);
  }
  bool write(const void* p, size_t bytes) { return bytes == 0 || std::fwrite(p, 1, bytes, f) == bytes; }
  bool read(void* p, size_t bytes) { return bytes == 0 || std::fread(p, 1, bytes, f) == bytes; }
  bool at_end() {
    const int c = std::fgetc(f);
    return c == EOF;
  }
};

// unshifted cell index of a particle (x fastest), the checkpoint order of mpc_get_state
inline uint64_t cell_of(uint32_t x, uint32_t y, uint32_t z, int F, const int L[3]) {
  return (uint64_t)(x >> F) + (uint64_t)L[0] * ((uint64_t)(y >> F) + (uint64_t)L[1] * (uint64_t)(z >> F));
}

mpc_status bad(const std::string& msg) { return fail(nullptr, MPC_EINVAL, "checkpoint: " + msg); }

}  // namespace

extern "C" {

mpc_status mpc_checkpoint_write(mpc_handle h, const char* prefix) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!prefix || !*prefix) return fail(h, MPC_EINVAL, "prefix is NULL or empty");
  if (!little_endian()) return fail(h, MPC_EINVAL, "checkpoints are little-endian");
  const int64_t N = h->N;
  const mpc_params& p = h->p;
  const int F = h->g.F;
  std::vector<uint32_t> X((size_t)N * 3), id((size_t)N);
  std::vector<float> V((size_t)N * 3);
  int64_t step = 0;
  TRY(mpc_get_state(h, X.data(), V.data(), id.data(), nullptr, &step, 0));
  const uint64_t C = (uint64_t)p.L[0] * p.L[1] * p.L[2];
  std::vector<uint32_t> count((size_t)C, 0);
  uint64_t prev = 0;
  for (int64_t i = 0; i < N; ++i) {
    const uint64_t c = cell_of(X[(size_t)i], X[(size_t)(N + i)], X[(size_t)(2 * N + i)], F, p.L);
    if (c >= C || c < prev) return fail(h, MPC_ESTATE, "checkpoint: state not ordered by cell");
    prev = c;
    count[(size_t)c] += 1;
  }
  const std::string base(prefix);
  {
    File t(base + ".txt", "w");
    if (!t.f) return fail(h, MPC_EINVAL, "cannot write " + base + ".txt");
    const int ok = std::fprintf(
        t.f,
        "format = mpc-checkpoint %d\nL = %d %d %d\na = %.17g\nn_c = %.17g\nh = %.17g\n"
        "alpha_deg = %.17g\nkT = %.17g\nm = %.17g\nvariant = %d\nthermostat = %d\nwalls_z = %d\n"
        "gravity = %.17g %.17g %.17g\nseed = %" PRIu64 "\nbox_id = %u\nflags = %u\nstep = %" PRId64
        "\nn_particles = %" PRId64 "\nfixed_bits = %d\ncells = %" PRIu64 "\noffset_bytes = %d\n"
        "wall_u = %.17g %.17g\n",
        kFormat, p.L[0], p.L[1], p.L[2], p.a, p.n_c, p.h, p.alpha_deg, p.kT, p.m, p.variant,
        p.thermostat, p.walls_z, p.gravity[0], p.gravity[1], p.gravity[2], p.seed, p.box_id, p.flags,
        step, N, F, C, N >= (1LL << 32) ? 8 : 4, p.wall_u[0], p.wall_u[1]);
    if (ok < 0) return fail(h, MPC_EINVAL, "cannot write " + base + ".txt");
  }
  {
    File b(base + ".particles", "wb");
    if (!b.f || !b.write(X.data(), X.size() * 4) || !b.write(V.data(), V.size() * 4) ||
        !b.write(id.data(), id.size() * 4))
      return fail(h, MPC_EINVAL, "cannot write " + base + ".particles");
  }
  {
    File c(base + ".cells", "wb");
    if (!c.f || !c.write(count.data(), count.size() * 4)) return fail(h, MPC_EINVAL, "cannot write " + base + ".cells");
    uint64_t off = 0;
    const bool wide = N >= (1LL << 32);
    std::vector<uint32_t> o32;
    std::vector<uint64_t> o64;
    (wide ? o64.resize((size_t)C) : o32.resize((size_t)C));
    for (uint64_t k = 0; k < C; ++k) {
      if (wide) o64[(size_t)k] = off;
      else o32[(size_t)k] = (uint32_t)off;
      off += count[(size_t)k];
    }
    const bool ok = wide ? c.write(o64.data(), o64.size() * 8) : c.write(o32.data(), o32.size() * 4);
    if (!ok) return fail(h, MPC_EINVAL, "cannot write " + base + ".cells");
  }
  return MPC_OK;
}

mpc_status mpc_checkpoint_read(const char* prefix, void* stream, const mpc_allocator* alloc,
                               mpc_handle* out) {
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (!prefix || !*prefix) return bad("prefix is NULL or empty");
  if (!little_endian()) return bad("checkpoints are little-endian");
  const std::string base(prefix);
  std::map<std::string, std::string> kv;
  {
    File t(base + ".txt", "r");
    if (!t.f) return bad("cannot open " + base + ".txt");
    char line[512];
    while (std::fgets(line, sizeof line, t.f)) {
      std::string s(line);
      const size_t eq = s.find('=');
      if (eq == std::string::npos) continue;
      auto trim = [](std::string v) {
        const size_t a = v.find_first_not_of(" \t\r\n"), b = v.find_last_not_of(" \t\r\n");
        return a == std::string::npos ? std::string() : v.substr(a, b - a + 1);
      };
      kv[trim(s.substr(0, eq))] = trim(s.substr(eq + 1));
    }
  }
  for (const char* k : {"format", "L", "a", "n_c", "h", "alpha_deg", "kT", "m", "variant", "thermostat",
                        "walls_z", "gravity", "seed", "box_id", "flags", "step", "n_particles",
                        "fixed_bits", "cells", "offset_bytes"})
    if (!kv.count(k)) return bad(std::string("missing key ") + k);
  int fmt = 0;
  if (std::sscanf(kv["format"].c_str(), "mpc-checkpoint %d", &fmt) != 1 || fmt != kFormat)
    return bad("unknown format " + kv["format"]);
  mpc_params p{};
  int64_t step = 0, N = 0;
  int F = 0, off_bytes = 0;
  uint64_t C = 0;
  bool ok = std::sscanf(kv["L"].c_str(), "%d %d %d", &p.L[0], &p.L[1], &p.L[2]) == 3 &&
            std::sscanf(kv["a"].c_str(), "%lf", &p.a) == 1 &&
            std::sscanf(kv["n_c"].c_str(), "%lf", &p.n_c) == 1 &&
            std::sscanf(kv["h"].c_str(), "%lf", &p.h) == 1 &&
            std::sscanf(kv["alpha_deg"].c_str(), "%lf", &p.alpha_deg) == 1 &&
            std::sscanf(kv["kT"].c_str(), "%lf", &p.kT) == 1 &&
            std::sscanf(kv["m"].c_str(), "%lf", &p.m) == 1 &&
            std::sscanf(kv["variant"].c_str(), "%d", &p.variant) == 1 &&
            std::sscanf(kv["thermostat"].c_str(), "%d", &p.thermostat) == 1 &&
            std::sscanf(kv["walls_z"].c_str(), "%d", &p.walls_z) == 1 &&
            std::sscanf(kv["gravity"].c_str(), "%lf %lf %lf", &p.gravity[0], &p.gravity[1], &p.gravity[2]) == 3 &&
            std::sscanf(kv["seed"].c_str(), "%" SCNu64, &p.seed) == 1 &&
            std::sscanf(kv["box_id"].c_str(), "%u", &p.box_id) == 1 &&
            std::sscanf(kv["flags"].c_str(), "%u", &p.flags) == 1 &&
            std::sscanf(kv["step"].c_str(), "%" SCNd64, &step) == 1 &&
            std::sscanf(kv["n_particles"].c_str(), "%" SCNd64, &N) == 1 &&
            std::sscanf(kv["fixed_bits"].c_str(), "%d", &F) == 1 &&
            std::sscanf(kv["cells"].c_str(), "%" SCNu64, &C) == 1 &&
            std::sscanf(kv["offset_bytes"].c_str(), "%d", &off_bytes) == 1;
  if (kv.count("wall_u") &&
      std::sscanf(kv["wall_u"].c_str(), "%lf %lf", &p.wall_u[0], &p.wall_u[1]) != 2)
    ok = false;
  if (!ok) return bad("malformed value in " + base + ".txt");
  for (int ax = 0; ax < 3; ++ax)
    if (p.L[ax] < 2 || p.L[ax] > 1024) return bad("L out of range");
  if (N < 1 || N != std::llround((double)p.L[0] * p.L[1] * p.L[2] * p.n_c))
    return bad("n_particles does not match L and n_c");
  if (F != mpc::fixed_bits_for(p.L)) return bad("fixed_bits does not match L");
  if (C != (uint64_t)p.L[0] * p.L[1] * p.L[2]) return bad("cells does not match L");
  if (off_bytes != (N >= (1LL << 32) ? 8 : 4)) return bad("offset_bytes does not match n_particles");
  if (step < 0) return bad("negative step");
  std::vector<uint32_t> X((size_t)N * 3), id((size_t)N);
  std::vector<float> V((size_t)N * 3);
  {
    File b(base + ".particles", "rb");
    if (!b.f || !b.read(X.data(), X.size() * 4) || !b.read(V.data(), V.size() * 4) ||
        !b.read(id.data(), id.size() * 4) || !b.at_end())
      return bad("particle file missing or of the wrong size");
  }
  std::vector<uint32_t> count((size_t)C);
  std::vector<uint64_t> offset((size_t)C);
  {
    File c(base + ".cells", "rb");
    if (!c.f || !c.read(count.data(), count.size() * 4)) return bad("cell file missing or short");
    if (off_bytes == 8) {
      if (!c.read(offset.data(), offset.size() * 8)) return bad("cell file short");
    } else {
      std::vector<uint32_t> o32((size_t)C);
      if (!c.read(o32.data(), o32.size() * 4)) return bad("cell file short");
      for (uint64_t k = 0; k < C; ++k) offset[(size_t)k] = o32[(size_t)k];
    }
    if (!c.at_end()) return bad("cell file too long");
  }
  // the counts and offsets must describe the particles' cells exactly
  uint64_t off = 0;
  for (uint64_t k = 0; k < C; ++k) {
    if (offset[(size_t)k] != off) return bad("cell offsets are not the prefix sums of the counts");
    off += count[(size_t)k];
  }
  if ((int64_t)off != N) return bad("cell counts do not add up to n_particles");
  const uint32_t P[3] = {(uint32_t)p.L[0] << F, (uint32_t)p.L[1] << F, (uint32_t)p.L[2] << F};
  for (uint64_t k = 0; k < C; ++k)
    for (uint64_t i = offset[(size_t)k]; i < offset[(size_t)k] + count[(size_t)k]; ++i) {
      const uint32_t x = X[(size_t)i], y = X[(size_t)(N + (int64_t)i)], z = X[(size_t)(2 * N + (int64_t)i)];
      if (x >= P[0] || y >= P[1] || z >= P[2]) return bad("a position lies outside the box");
      if (cell_of(x, y, z, F, p.L) != k) return bad("a particle is not in the cell its offsets give");
    }
  mpc_handle h = nullptr;
  TRY(mpc_create(&p, stream, alloc, &h));
  const mpc_status st = mpc_set_state(h, X.data(), V.data(), id.data(), step, 0);
  if (st != MPC_OK) {
    const std::string msg = h->err;
    mpc_destroy(h);
    return fail(nullptr, st, "checkpoint: " + msg);
  }
  *out = h;
  return MPC_OK;
}

}  // extern "C"
