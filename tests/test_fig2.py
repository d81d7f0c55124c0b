"""Fig. 2's accuracy claims on the CPU oracle, in the paper's setting (Sec. V): against REF =
BENR at 1e-14 s, on an inverter output of a switching inverter chain, ER at 1e-13 s is more
accurate than BENR at 1e-13 s, and ER-C at twice that step still is."""
from fig2_study import paper_setting


def test_fig2_er_and_erc_beat_benr():
    node, errs = paper_setting()
    be = errs["BENR 0.1 ps"][0]
    assert errs["ER 0.1 ps"][0] < be / 4, errs
    assert errs["ER-C 0.2 ps"][0] < be, errs
    # second order against first: halving ER's step cuts its error about 4x
    assert 2.5 < errs["ER 0.2 ps"][1] / errs["ER 0.1 ps"][1] < 6.0, errs
