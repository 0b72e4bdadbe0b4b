"""Writes the value column of panel_closed_forms.txt from the hand derivations
in that file's header (plain `math`, no oracle or library code involved)."""
import math

VALUES = [
    ("-1 0 1 0 0 0 0 S", 1.0 / math.pi),
    ("-1 0 1 0 0 1 0 S", -(math.log(2) - 2 + math.pi / 2) / (2 * math.pi)),
    ("-1 0 1 0 0 0 1 S", -(math.log(2) - 2 + math.pi / 2) / (2 * math.pi)),
    ("-1 0 1 0 -1 0 0 S", (1 - math.log(2)) / math.pi),
    ("-1 0 1 0 0 1 0 Dl", -0.25),
    ("-1 0 1 0 0 -1 0 Dl", 0.25),
    ("-1 0 1 0 0 1 0 dS/dbx", -math.log(2) / (4 * math.pi)),
    ("-1 0 1 0 0 1 0 dS/dby", 0.125),
    ("-1 0 1 0 0 1 0 dDl/dbx", -1.0 / (4 * math.pi)),
    ("-1 0 1 0 0 1 0 dDl/dby", -1.0 / (4 * math.pi)),
]

if __name__ == "__main__":
    for key, v in VALUES:
        print(f"{key} {v:.17g}")
