// partition.cpp -- exchange plan of a partitioned context: the boundary strips that processes
// owning different ranges of sub-domains (the paper's PEs, Sec. 3) send each other.
//
// In the paper every PE sends the boundary strips of its new solution to its neighbours and
// receives theirs into its multi-level buffers (Alg. 1-3).  Here a process computes a contiguous
// range of sub-domains and keeps state arrays of the whole grid; the points of other processes'
// sub-domains that its own sub-domains read -- the halo of the difference stencils (faces to the
// halo depth, viscous edges to r x r) and of the filter lines (faces to depth 5) -- arrive through
// the exchange, everything else of a foreign sub-domain is never read.  On a connected grid a
// point beyond a non-periodic block face is read through its gather entry (an interface
// neighbour's points, interpolated spanwise; the mirror point of a wall; the face point of an
// outflow), so the sources of those entries join the lists.  Both sides derive the lists from the
// same decomposition in the same order, so a list can be sent as a plain array of values with no
// indices.
#include <algorithm>
#include <vector>

#include "cfs_internal.h"

namespace cfs {

namespace {

// Sub-domain origin and length along an axis of n points split into p parts (the first n mod p
// parts one point longer), as cfs_split_block defines it.
void split(int n, int p, int i, int* o, int* s) {
  const int q = n / p, rem = n % p;
  *s = q + (i < rem ? 1 : 0);
  *o = i * q + std::min(i, rem);
}

int wrap(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

}  // namespace

const char* strip_plan(const TopoBlock* B, int nb, int nsub, const int* starts, int nranks, int rank, int depth,
                       int depth_z, int r, bool viscous, int ndim, StripPlan* out) {
  if (nranks < 1 || rank < 0 || rank >= nranks || !starts) return "bad partition";
  if (starts[0] != 0 || starts[nranks] != nsub) return "the partition must cover sub-domains 0 .. nsub - 1";
  for (int q = 0; q < nranks; ++q)
    if (starts[q + 1] < starts[q]) return "partition boundaries must not decrease";
  std::vector<int> rank_of(nsub);
  for (int q = 0; q < nranks; ++q)
    for (int s = starts[q]; s < starts[q + 1]; ++s) rank_of[s] = q;
  // per block and axis: the sub-domain index along the axis of every coordinate
  std::vector<std::vector<int>> owner((size_t)nb * 3);
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      std::vector<int>& ow = owner[(size_t)b * 3 + a];
      ow.resize(B[b].n[a]);
      for (int i = 0; i < B[b].P[a]; ++i) {
        int o, s;
        split(B[b].n[a], B[b].P[a], i, &o, &s);
        for (int t = 0; t < s; ++t) ow[o + t] = i;
      }
    }
  std::vector<std::vector<long long>> send(nranks), recv(nranks);
  std::vector<std::vector<int>> send_n(nranks), recv_n(nranks);
  for (int b = 0; b < nb; ++b) {
    const TopoBlock& T = B[b];
    const bool per = topo_periodic(T);
    const int n3[3] = {T.n[0], T.n[1], T.n[2]};
    for (int iz = 0; iz < T.P[2]; ++iz)
      for (int iy = 0; iy < T.P[1]; ++iy)
        for (int ix = 0; ix < T.P[0]; ++ix) {
          const int sid = T.sid0 + ix + T.P[0] * (iy + T.P[1] * iz);
          const int p = rank_of[sid];
          int o[3], sz[3];
          split(n3[0], T.P[0], ix, &o[0], &sz[0]);
          split(n3[1], T.P[1], iy, &o[1], &sz[1]);
          split(n3[2], T.P[2], iz, &o[2], &sz[2]);
          const int dep[3] = {depth, depth, ndim == 3 ? depth_z : 0};
          // the read set: points within dep[a] beyond one face (inside the sub-domain along the
          // other axes), and for viscous runs points within r beyond two faces (edges)
          for (int dk = -dep[2]; dk < sz[2] + dep[2]; ++dk)
            for (int dj = -dep[1]; dj < sz[1] + dep[1]; ++dj)
              for (int di = -dep[0]; di < sz[0] + dep[0]; ++di) {
                const int c[3] = {di, dj, dk};
                int nout = 0, far = 0;
                for (int a = 0; a < 3; ++a) {
                  const int d = c[a] < 0 ? -c[a] : (c[a] >= sz[a] ? c[a] - sz[a] + 1 : 0);
                  if (d > 0) ++nout;
                  if (d > r) far = 1;
                }
                if (nout == 0 || nout == 3) continue;
                if (nout == 2 && (!viscous || far)) continue;
                auto add = [&](long long off, int bN, int q) {
                  if (q == p) return;
                  if (p == rank) {
                    recv[q].push_back(off);
                    recv_n[q].push_back(bN);
                  } else if (q == rank) {
                    send[p].push_back(off);
                    send_n[p].push_back(bN);
                  }
                };
                bool beyond = false;  // beyond a non-periodic face of the block
                for (int a = 0; a < 3; ++a) {
                  const int x = o[a] + c[a];
                  if ((x < 0 && T.face[2 * a].type != FACE_PERIODIC) || (x >= n3[a] && T.face[2 * a + 1].type != FACE_PERIODIC))
                    beyond = true;
                }
                if (!per && beyond) {
                  GatherEntry e;
                  if (!gather_entry(B, nb, b, o[0] + c[0], o[1] + c[1], o[2] + c[2], &e))
                    return "a point beyond a block face does not resolve";
                  for (int t = 0; t < e.nt; ++t) add(e.off[t], e.bN[t], rank_of[e.sid[t]]);
                  continue;
                }
                int gc[3], oc[3];
                for (int a = 0; a < 3; ++a) {
                  gc[a] = wrap(o[a] + c[a], n3[a]);
                  oc[a] = owner[(size_t)b * 3 + a][gc[a]];
                }
                const int src = T.sid0 + oc[0] + T.P[0] * (oc[1] + T.P[1] * oc[2]);
                const long long off = T.base + (long long)gc[0] + (long long)n3[0] * ((long long)gc[1] + (long long)n3[1] * gc[2]);
                add(off, (int)T.N, rank_of[src]);
              }
        }
  }
  // sorted, without repeats (a point read by several sub-domains travels once); the block size
  // follows the offset (blocks are stored one after another)
  auto finish = [&](std::vector<std::vector<long long>>& L, std::vector<std::vector<int>>& Ln, std::vector<long long>& offs,
                    std::vector<long long>& flat, std::vector<int>& flat_n) {
    offs.assign(nranks + 1, 0);
    flat.clear();
    flat_n.clear();
    for (int q = 0; q < nranks; ++q) {
      std::vector<std::pair<long long, int>> v(L[q].size());
      for (size_t i = 0; i < v.size(); ++i) v[i] = {L[q][i], Ln[q][i]};
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      for (auto& e : v) {
        flat.push_back(e.first);
        flat_n.push_back(e.second);
      }
      offs[q + 1] = (long long)flat.size();
    }
  };
  finish(send, send_n, out->send_off, out->send, out->send_bN);
  finish(recv, recv_n, out->recv_off, out->recv, out->recv_bN);
  return nullptr;
}

}  // namespace cfs
