"""Per-level records of a V-cycle (Algorithm 1 with label propagation on
every level) for the exact-parity tests: sizes, SHA-256 digests of the
canonical level CSR, of the map to the next level and of the partition
after label propagation, plus objectives and moves.  `gpu_records` runs the
steps through the C ABI; `oracle_records` turns an oracle V-cycle into the
same form.  Digests are over little-endian int32 bytes."""
import hashlib

import numpy as np


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def gpu_records(hg, torch, hgr, k, eps, passes, opt, device_input=True):
    stream = torch.cuda.current_stream()
    if device_input:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
        h = hg.hg_create(hgr.n, hgr.m, t(hgr.offsets), t(hgr.pins), t(hgr.net_w), t(hgr.node_w),
                         hg.HG_MEM_DEVICE, opt, stream)
    else:
        h = hg.hg_create(hgr.n, hgr.m, hgr.offsets, hgr.pins, hgr.net_w, hgr.node_w,
                         hg.HG_MEM_HOST, opt, stream)
    try:
        while hg.hg_coarsen_level(h, k)[0] == hg.HG_OK:
            pass
        nl = hg.hg_num_levels(h)
        recs = []
        for lv in range(nl):
            got = hg.hg_get_level(h, lv, with_map=lv < nl - 1)
            n, m, p = hg.hg_level_info(h, lv)
            rec = {"n": n, "m": m, "p": p, "offsets": digest(got["offsets"]),
                   "pins": digest(got["pins"]), "net_w": digest(got["net_w"]),
                   "node_w": digest(got["node_w"]), "graph": hg.hg_level_is_graph(h, lv)}
            if lv < nl - 1:
                rec["map"] = digest(got["map"])
            recs.append(rec)
        top = nl - 1
        parts = [torch.empty(max(recs[lv]["n"], 1), dtype=torch.int32, device="cuda")
                 for lv in range(nl)]
        hg.hg_initial_partition(h, top, k, parts[top])
        initial = hg.hg_objective(h, top, k, parts[top])
        for lv in range(top, -1, -1):
            if lv < top:
                hg.hg_project(h, lv + 1, parts[lv + 1], parts[lv])
            obj, moves = hg.hg_lp_refine(h, lv, k, eps, passes, parts[lv])
            recs[lv]["objective"] = obj
            recs[lv]["moves"] = moves
            recs[lv]["part"] = digest(parts[lv][:recs[lv]["n"]].cpu().numpy())
        return recs, initial
    finally:
        hg.hg_destroy(h)


def oracle_records(vc):
    out = []
    for lv, L in enumerate(vc.levels):
        w = {"n": int(L.n), "m": int(L.m), "p": int(L.p), "offsets": digest(L.offsets),
             "pins": digest(L.pins), "net_w": digest(L.net_w), "node_w": digest(L.node_w),
             "part": digest(vc.parts[lv]), "objective": int(vc.objectives[lv]),
             "moves": int(vc.moves[lv])}
        if lv < len(vc.maps):
            w["map"] = digest(vc.maps[lv])
        out.append(w)
    return out


KEYS = ("n", "m", "p", "offsets", "pins", "net_w", "node_w", "map", "objective", "moves", "part")


def compare_records(got, want):
    assert len(got) == len(want), f"levels: gpu {len(got)} vs oracle {len(want)}"
    for lv, (g, w) in enumerate(zip(got, want)):
        for key in KEYS:
            if key in w:
                assert g.get(key) == w[key], (
                    f"level {lv}: {key} differs (gpu {g.get(key)}, oracle {w[key]})")
