"""GPU parity of ms_training_records (walk records -> CVAE conditions and targets, Sec. 4.1) with the
oracle transform.  Both sides receive the same records, produced by the oracle walk."""
import numpy as np
import pytest
import torch

from oracle import cvae
from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu


def test_training_records_match_oracle(orc):
    n = 20000
    tau, g, phi = synth.training_media(4, n)
    tau = np.minimum(tau, 40.0).astype(np.float32)
    g, phi = g.astype(np.float32), phi.astype(np.float32)
    r = orc.walk(2, n, dict(optical_radius=tau.astype(np.float64), g=g.astype(np.float64),
                            albedo=phi.astype(np.float64), dir_in=(0.0, 0.0, 1.0), isotropic_start=0,
                            first_event_at_origin=1), reservoir_mode=2)
    f32 = {k: r[k].astype(np.float32) for k in ("exit_pos", "exit_dir", "rep_pos", "rep_dir")}
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    media = ms.media_tensor(tau, g, phi, (0, 0, 1), 0, 1)
    recs = {k: torch.zeros(n, d, device="cuda") for k, d in
            (("cL", 2), ("xL", 1), ("cP", 3), ("xP", 3), ("cE", 7), ("xE", 6))}
    ms.ms_training_records(n, dev(r["n_events"]), dev(f32["exit_pos"]), dev(f32["exit_dir"]), dev(f32["rep_pos"]),
                           dev(f32["rep_dir"]), media, 9, recs)
    torch.cuda.synchronize()
    u = orc.u24(orc.philox_words(9, 0, n, 0, 0x44)[:, 0])
    ref = cvae.training_targets(r["n_events"], *(f32[k].astype(np.float64) for k in
                                                 ("exit_pos", "exit_dir", "rep_pos", "rep_dir")), tau, g, phi, u)
    for k, v in recs.items():
        got = v.cpu().numpy()
        assert np.abs(got - ref[k]).max() <= 2e-5 * max(1.0, np.abs(ref[k]).max()), k
