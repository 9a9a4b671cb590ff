"""Write tests/golden/lp_objectives.json: the optimum of the centralized LP
(Eq. LP_model) of each configuration feeder, solved by HiGHS through the
oracle.  Calls only oracle/ (and the seeded feeder generator).

    python tests/golden/make_lp_objectives.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lp as OL, model as OM          # noqa: E402
from paper_2501_08293_b300 import feeders as F     # noqa: E402


def main():
    out = {"_source": "HiGHS (scipy linprog) on the LP of Eq. (LP_model) built by oracle/model.py",
           "feeders": {}}
    for name, f in (("13", F.feeder_13(1)), ("123", F.feeder_123(1)), ("8500", F.feeder_8500(1))):
        t = time.time()
        m = OM.build_feeder(f)
        r = OL.solve_lp(m)
        out["feeders"][name] = {"feeder": f.name, "status": int(r.status), "objective": float(r.fun),
                                "n_global": m.n, "seconds": round(time.time() - t, 2)}
        print(name, out["feeders"][name], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lp_objectives.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
