"""What the trained vetter gains over the method without it.

Forty seeded training fields (decam_tno geometry, uneven epochs and noise,
magnitudes extended to p = 0.06) are searched at the lowered threshold
n_low(E); the ownership-selected candidates' stamps train the CNN on the GPU
(the library's forward, backward and Adam kernels).  Ten further fields fix
the logit threshold for a purity of 0.95.  On twelve held-out fields:

  * recall per 0.5-mag bin of the vetted form is at least the plain
    threshold's (N_min = ceil(E/4)) in every bin, and far higher in the two
    faintest bins (movers with too few detections for the plain threshold);
  * the network is what makes the lowered threshold usable: without it the
    owned candidates are mostly noise alignments (purity ~ 0.2), with it the
    purity is >= 0.9.
"""
import numpy as np
import pytest

from paper_2509_26279_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_26279_gb300 import sas, vetting  # noqa: E402


def test_trained_vetter_beats_plain_threshold():
    dev = torch.device("cuda", 0)
    train_fields = W.vetter_fields(40, seed=W.BASE_SEED + 50)
    eval_fields = W.vetter_fields(12, seed=W.BASE_SEED + 60)
    st, lab = vetting.training_set(train_fields, dev)
    assert st.shape[0] > 20000 and 0.05 < float(lab.mean()) < 0.5
    vt = sas.Vetter(0, 512)
    vt.set_state(vetting.init_params(1))
    hist = vetting.train(vt, st, lab, epochs=20, batch=512, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    cst, clab = vetting.training_set(W.vetter_fields(10, seed=W.BASE_SEED + 70), dev)
    tau = vetting.calibrate(vetting.logits_of(vt, cst), clab.cpu().numpy(), 0.95)
    assert np.isfinite(tau)
    r = vetting.evaluate(vt, eval_fields, dev, threshold=tau)
    plain, owned, vetted = r["plain"], r["owned"], r["vetted"]
    print({"tau": tau, **{k: (r[k]["purity"], r[k]["recall"]) for k in ("plain", "low", "owned", "vetted")}})
    for b in range(len(plain["total"])):
        assert vetted["found"][b] >= plain["found"][b] - 3, (b, vetted["found"], plain["found"])
    for b in (-2, -1):
        assert vetted["recall"][b] >= plain["recall"][b] + 0.25, (vetted["recall"], plain["recall"])
    assert vetted["purity"] >= 0.9, vetted["purity"]
    assert owned["purity"] <= 0.5 and vetted["purity"] >= owned["purity"] + 0.4
