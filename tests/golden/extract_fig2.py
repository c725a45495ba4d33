"""Write the Fig. 2 fixtures of the paper as plain text.

Fig. 2 of "Fast Isotopy Computation for T-Curves" prints three degree-8
triangulations (first quadrant, as TikZ edge drawings) and, for each, the
percentage of the 2^42 sign-distribution classes whose curve has k ovals
(as a PGF ``const plot``; the bin of k ovals is the coordinate x = k - 0.5).
This script reads the paper's LaTeX source and writes:

  fig2_<name>.edges          one edge "i1 j1 i2 j2" per line
  fig2_oval_percentages.txt  "<name> <k> <percent>" per line

Run it by hand with the path of the paper's LaTeX source:
    python tests/golden/extract_fig2.py <paper source>
"""
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ("bow_tie", "rank016", "rank015")


def sections(text):
    parts = re.split(r"^%% file: (\S+)\s*$", text, flags=re.M)
    return {parts[k]: parts[k + 1] for k in range(1, len(parts) - 1, 2)}


def main(path):
    sec = sections(open(path, encoding="utf-8").read())
    rows = []
    for name in NAMES:
        wire = sec[f"tikz/{name}_wireframe.tex"]
        edges = re.findall(r"\\draw\[[^\]]*\]\s*\((\d+),(\d+)\)\s*--\s*\((\d+),(\d+)\);", wire)
        with open(os.path.join(HERE, f"fig2_{name}.edges"), "w") as f:
            f.write(f"# Fig. 2 of the paper, triangulation '{name}' of 8*Delta_2 "
                    f"(TikZ wireframe data): one edge i1 j1 i2 j2 per line\n")
            for e in edges:
                f.write(" ".join(e) + "\n")
        hist = sec[f"tikz/{name}_histogram.tex"]
        for x, y in re.findall(r"\((-?\d+\.5),([\d.]+)\)", hist):
            k = int(round(float(x) + 0.5))
            rows.append((name, k, y))
    with open(os.path.join(HERE, "fig2_oval_percentages.txt"), "w") as f:
        f.write("# Fig. 2 of the paper: percent of the 2^42 sign-distribution classes "
                "with k ovals (const-plot bin x = k - 0.5)\n")
        for name, k, y in rows:
            if k <= 22:
                f.write(f"{name} {k} {y}\n")


if __name__ == "__main__":
    main(sys.argv[1])
