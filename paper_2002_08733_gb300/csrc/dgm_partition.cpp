// Element partitions for running one mesh on several GPUs (host code).
//
// The right-hand side of an element (Secs. III-IV) reads only its own
// coefficients and those of its face neighbours, so a partition of the
// elements needs one exchange per stage: every part receives the current
// coefficients of the other parts' elements that touch it through a face (its
// halo) before it evaluates the next stage.
//
// dgm_partition_slabs cuts the mesh into slabs along one axis: elements sorted
// by centroid coordinate (ties by element id), split into contiguous runs of
// nearly equal size.  On a Kuhn grid these are k-plane slabs, and each part
// talks to at most two others.
//
// dgm_halo_build gives one part its local numbering -- owned elements first,
// then halo (ghost) elements, each in ascending global id -- and, per peer
// part, the local ids it sends and the local ids it receives into.  Both
// sides list the elements of a peer pair in ascending global id, so a send
// list and the matching receive list on the peer line up entry by entry.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "dgm_internal.h"
#include "dgmax.h"

namespace dgm {
int partition_fail(int code, const std::string& msg);   // sets the thread's last error (dgm_api.cu)
}

using namespace dgm;

extern "C" int dgm_partition_slabs(int64_t nv, const double* xyz, int64_t nt, const int64_t* tets,
                                   int32_t axis, int32_t nparts, int32_t* part) {
    if (nv < 1 || nt < 1 || !xyz || !tets || !part) return partition_fail(DGM_EINVAL, "empty mesh or null input");
    if (axis < 0 || axis > 2) return partition_fail(DGM_EINVAL, "axis must be 0, 1 or 2");
    if (nparts < 1 || int64_t(nparts) > nt)
        return partition_fail(DGM_EINVAL, "need 1 <= nparts <= number of elements");
    std::vector<std::pair<double, int64_t>> key(static_cast<size_t>(nt));
    for (int64_t e = 0; e < nt; ++e) {
        double c = 0.0;
        for (int i = 0; i < 4; ++i) {
            const int64_t v = tets[4 * e + i];
            if (v < 0 || v >= nv) return partition_fail(DGM_EMESH, "vertex id out of range in element " + std::to_string(e));
            c += xyz[3 * v + axis];
        }
        key[size_t(e)] = {0.25 * c, e};
    }
    std::sort(key.begin(), key.end());
    for (int64_t i = 0; i < nt; ++i)   // part r gets sorted positions [r nt / P, (r+1) nt / P)
        part[key[size_t(i)].second] = int32_t((i * int64_t(nparts)) / nt);
    return DGM_OK;
}

extern "C" int dgm_halo_build(int64_t nt, const int64_t* tets, const int32_t* part, int32_t nparts,
                              int32_t rank, dgm_halo_sizes* sizes, int64_t* local_to_global,
                              int32_t* peers, int64_t* send_count, int64_t* send_idx,
                              int64_t* recv_count, int64_t* recv_idx) {
    if (nt < 1 || !tets || !part || !sizes) return partition_fail(DGM_EINVAL, "empty mesh or null input");
    if (nparts < 1 || rank < 0 || rank >= nparts) return partition_fail(DGM_EINVAL, "rank out of range");
    for (int64_t e = 0; e < nt; ++e)
        if (part[e] < 0 || part[e] >= nparts) return partition_fail(DGM_EINVAL, "part id out of range");
    // face adjacency by sorted vertex triples
    struct FaceKey {
        std::array<int64_t, 3> v;
        int64_t e;
    };
    std::vector<FaceKey> faces;
    faces.reserve(size_t(4 * nt));
    for (int64_t e = 0; e < nt; ++e) {
        std::array<int64_t, 4> s = {tets[4 * e], tets[4 * e + 1], tets[4 * e + 2], tets[4 * e + 3]};
        std::sort(s.begin(), s.end());
        for (int f = 0; f < 4; ++f) {
            std::array<int64_t, 3> t;
            int c = 0;
            for (int i = 0; i < 4; ++i)
                if (i != f) t[c++] = s[i];
            faces.push_back({t, e});
        }
    }
    std::sort(faces.begin(), faces.end(), [](const FaceKey& a, const FaceKey& b) {
        return a.v != b.v ? a.v < b.v : a.e < b.e;
    });
    // owned elements adjacent to each peer (sent to it), peers' elements adjacent to us (ghosts)
    std::map<int32_t, std::vector<int64_t>> send, recv;
    for (size_t i = 0; i + 1 < faces.size(); ++i) {
        if (faces[i].v != faces[i + 1].v) continue;
        const int64_t a = faces[i].e, b = faces[i + 1].e;
        if (part[a] == part[b]) continue;
        if (part[a] == rank) {
            send[part[b]].push_back(a);
            recv[part[b]].push_back(b);
        } else if (part[b] == rank) {
            send[part[a]].push_back(b);
            recv[part[a]].push_back(a);
        }
    }
    for (auto* m : {&send, &recv})
        for (auto& kv : *m) {
            std::sort(kv.second.begin(), kv.second.end());
            kv.second.erase(std::unique(kv.second.begin(), kv.second.end()), kv.second.end());
        }
    std::vector<int64_t> owned, ghosts;
    for (int64_t e = 0; e < nt; ++e)
        if (part[e] == rank) owned.push_back(e);
    for (auto& kv : recv) ghosts.insert(ghosts.end(), kv.second.begin(), kv.second.end());
    std::sort(ghosts.begin(), ghosts.end());
    sizes->n_owned = int64_t(owned.size());
    sizes->n_ghost = int64_t(ghosts.size());
    sizes->n_peers = int32_t(send.size());
    int64_t ns = 0, nr = 0;
    for (auto& kv : send) ns += int64_t(kv.second.size());
    for (auto& kv : recv) nr += int64_t(kv.second.size());
    sizes->n_send = ns;
    sizes->n_recv = nr;
    if (!local_to_global) return DGM_OK;   // sizes only
    if (!peers || !send_count || !send_idx || !recv_count || !recv_idx)
        return partition_fail(DGM_EINVAL, "null output array");
    std::map<int64_t, int64_t> g2l;
    for (size_t i = 0; i < owned.size(); ++i) {
        local_to_global[i] = owned[i];
        g2l[owned[i]] = int64_t(i);
    }
    for (size_t j = 0; j < ghosts.size(); ++j) {
        local_to_global[owned.size() + j] = ghosts[j];
        g2l[ghosts[j]] = int64_t(owned.size() + j);
    }
    int q = 0;
    int64_t is = 0, ir = 0;
    for (auto& kv : send) {
        peers[q] = kv.first;
        send_count[q] = int64_t(kv.second.size());
        for (int64_t g : kv.second) send_idx[is++] = g2l[g];
        const auto& rv = recv[kv.first];
        recv_count[q] = int64_t(rv.size());
        for (int64_t g : rv) recv_idx[ir++] = g2l[g];
        ++q;
    }
    return DGM_OK;
}
