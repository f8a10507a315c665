"""The landmark layout and run tables that povar_create builds on the
device, against a numpy construction from their stated rules (integer work:
bit-exact). Rules: observations of a landmark in camera order (stable sort
by camera, then by landmark); landmarks sorted by (smallest camera, longest
track first), ties by landmark id; every smallest camera starts a new slice
(its last slice padded to 32 slots); all slices ordered by width (longest
track, widest first, stable); padding to a multiple of 256 slots; entry (slice s, row t, lane l) at sell_off[s] + 32 t
+ l; a slice row is uniform (mask 0, one partial) when its valid lanes share
one camera, else bit l marks a lane whose camera differs from lane l - 1's
and every such lane with a valid camera opens a partial; partials are
numbered row by row and listed per camera in increasing index."""
import numpy as np
import pytest

from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF


def expected_layout(sc):
    cam = sc.cam_idx.astype(np.int64)
    pt = sc.pt_idx.astype(np.int64)
    np_, nc = sc.n_points, sc.n_cams
    by_cam = np.argsort(cam, kind="stable")
    perm = by_cam[np.argsort(pt[by_cam], kind="stable")]
    off = np.concatenate([[0], np.cumsum(np.bincount(pt, minlength=np_))])
    lens = np.diff(off)
    mincam = np.full(np_, np.iinfo(np.int64).max)
    np.minimum.at(mincam, pt, cam)
    maxlen = int(lens.max())
    assert int(maxlen).bit_length() + int(nc - 1).bit_length() <= 32
    order = np.lexsort((maxlen - lens, mincam))          # primary mincam, stable
    seq = []                                              # bucket-aligned sequence
    for c in np.unique(mincam):
        b = [int(j) for j in order if mincam[j] == c]
        seq += b + [NONE] * (-len(b) % 32)
    nseq = len(seq) // 32
    width_seq = np.array([max([lens[j] for j in seq[32 * s:32 * s + 32] if j != NONE])
                          for s in range(nseq)], dtype=np.int64)
    sl_order = np.argsort(-width_seq, kind="stable")
    np_pad = (len(seq) + 255) // 256 * 256
    slot_pt = np.full(np_pad, NONE, np.uint64)
    for s in range(nseq):
        slot_pt[32 * s:32 * s + 32] = seq[32 * sl_order[s]:32 * sl_order[s] + 32]
    nsl = np_pad // 32
    slot_len = np.array([lens[j] if j != NONE else 0 for j in slot_pt], np.int64)
    widths = slot_len.reshape(nsl, 32).max(axis=1)
    sell_off = np.concatenate([[0], np.cumsum(32 * widths)]).astype(np.int64)
    sell_cam = np.full(int(sell_off[-1]), -1, np.int64)
    for q in range(np_pad):
        j = int(slot_pt[q])
        if j == NONE:
            continue
        s, l = divmod(q, 32)
        for t in range(lens[j]):
            sell_cam[sell_off[s] + 32 * t + l] = cam[perm[off[j] + t]]
    nrows = len(sell_cam) // 32
    mask = np.zeros(nrows, np.int64)
    base = np.zeros(nrows, np.int64)
    pcam = []
    for r in range(nrows):
        c = sell_cam[32 * r:32 * r + 32]
        valid = c[c >= 0]
        base[r] = len(pcam)
        if len(valid) and np.all(valid == valid[0]):
            pcam.append(int(valid[0]))
            continue
        m = 0
        for l in range(32):
            if l == 0 or c[l] != c[l - 1]:
                m |= 1 << l
                if c[l] >= 0:
                    pcam.append(int(c[l]))
        mask[r] = m
    pcam = np.array(pcam, np.int64)
    pidx = np.argsort(pcam, kind="stable")
    poff = np.concatenate([[0], np.cumsum(np.bincount(pcam, minlength=nc))])
    return dict(slot_pt=slot_pt, sell_off=sell_off, sell_cam=sell_cam, row_mask=mask,
                row_base=base, cam_part_off=poff, cam_part_idx=pidx)


def ragged():
    base = scenes.ring_scene(13, 77, 21, track="uniform3to6", noise_px=1.0, eta=0.2)
    keep = base.cam_idx != 5   # a camera without observations
    return scenes.Scene(name="ragged", seed=21, n_cams=13, n_points=77,
                        cam_idx=base.cam_idx[keep].copy(), pt_idx=base.pt_idx[keep].copy(),
                        meas=base.meas[keep].copy(), eta=0.2, m=8, gt_cams=base.gt_cams,
                        gt_points=base.gt_points)


CASES = {
    "tiny": lambda: scenes.tiny_scene(0),
    "mid": lambda: scenes.mid_scene(0),
    "traj": lambda: scenes.trajectory_scene(120, 6000, 3, eta=0.1, m=8, name="traj"),
    "long": lambda: scenes.trajectory_scene(90, 2000, 8, eta=0.1, m=8, p_geom=0.03,
                                            max_track=70, outlier_frac=0.0, name="long"),
    "ragged": ragged,
}


@pytest.mark.parametrize("name", list(CASES))
def test_layout_and_run_tables_bit_exact(name):
    sc = CASES[name]()
    if name == "ragged" and np.bincount(sc.pt_idx, minlength=sc.n_points).min() == 0:
        pytest.skip("a landmark lost all its observations")
    exp = expected_layout(sc)
    with povar.Problem.from_scene(sc) as pb:
        got = pb.layout()
    for k, v in exp.items():
        assert np.array_equal(got[k].astype(np.int64), v.astype(np.int64)), k
